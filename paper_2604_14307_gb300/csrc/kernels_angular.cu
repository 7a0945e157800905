// Angular-momentum-conserving variants of the collision rules for the solvent
// (SRD+a and MPCD-AT+a: the modification of the rules that Sec. II.A of
// arXiv 2604.14307 cites from Noguchi and Gompper).
//
// After the plain rule has produced v*, every cell with two or more members
// gets the rigid rotation v' = v* + w x r_c that gives back its angular
// momentum about its centre of mass:
//     Pi w = sum_i m r_c,i x (v_i - v*_i),
// Pi the inertia tensor of the members about that centre, and w the least-norm
// solution when the members are collinear (two members in particular).  The
// rule conserves the momentum, so the correction keeps it as well.  r_c is
// measured on the 2^-20 lattice of the binning rule: Q = (floor(x 2^20) - S)
// mod 2^20 is the member's offset inside its shifted cell in units of 2^-20,
// an integer, which makes the geometric sums exact.
//
// Passes around the plain collision of a step (all keyed on the same step):
//   k_ang_sums<PRE>   before the rule: count, sum Q, sum Q_a Q_b, + sum Q x P, + sum P
//   k_ang_sums<POST>  after it:                                  - sum Q x P*, - sum P*
//   k_ang_params      per cell: centre, Pi and the angular-momentum change in
//                     FP64, w by Cholesky (least-norm form for collinear
//                     members); clears the words for the next collision
//   k_ang_apply       v = v* + w' x (N Q - sum Q),  w' = w / (N 2^20)
// The offset from the centre is formed as the exact integer N Q - sum Q: for
// nearly collinear members w is large along their line while the offsets
// across it are small, and an offset rounded in the working precision would
// carry an error of order eps |w| into the velocity.
// Word layout, SoA [ANG_WORDS][n_cells]:
//   0 N; 1-3 sum Q; 4-9 sum Q_a Q_b (xx, yy, zz, xy, xz, yz);
//   10-12 sum Q x (P - P*); 13-15 sum (P - P*).
// P32: P = round(fl32(m v) 2^20), the momentum term of the plain cell words,
// and every word an int64 sum (exact and independent of the order of the
// atomics; wrap-around of partial sums cancels as long as the final sum lies
// within +-2^63).  P64: P = m v in double; the Q sums are exact integers in
// double, the momentum sums FP64 atomics.
// The solvent mass is uniform, so Pi = m 2^-40 (tr(C) I - C) with C the
// lattice covariance sum Q_a Q_b - sum Q_a sum Q_b / N.
#include <algorithm>

#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

template <typename Real> struct AngWord;
template <> struct AngWord<float> { typedef long long type; };
template <> struct AngWord<double> { typedef double type; };

__device__ __forceinline__ void ang_red(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
__device__ __forceinline__ void ang_red(double *p, double v) { atomicAdd(p, v); }

// X = floor(x 2^20) of the binning rule, as in the plain passes (box edges
// below 2048 cells keep it within int32)
__device__ __forceinline__ int lattice_X(float x) { return __float2int_rd(x * 1048576.0f); }
__device__ __forceinline__ int lattice_X(double x) { return __double2int_rd(x * 1048576.0); }

__device__ __forceinline__ int axis_cell(int X, int S, int L)
{
    int c = (X - S) >> 20;
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    return ((unsigned)c < (unsigned)L) ? c : 0;   // only a non-finite position gets here
}

// momentum term P of one particle: the P32 fixed-point value or the FP64 product
__device__ __forceinline__ long long mom_term(float m, float v) { return q20(__fmul_rn(m, v)); }
__device__ __forceinline__ double mom_term(double m, double v) { return m * v; }

template <typename Real> __device__ __forceinline__ Real solvent_mass(const StepArgs &a);
template <> __device__ __forceinline__ float solvent_mass<float>(const StepArgs &a) { return a.m_solvent_f; }
template <> __device__ __forceinline__ double solvent_mass<double>(const StepArgs &a) { return a.m_solvent; }

struct TileFrame {
    int32_t L[3];
    int32_t S[3];
    int32_t base;
    int64_t beg, end;
};

__device__ __forceinline__ void load_frame(const StepArgs &a, int t, int64_t step, TileFrame &f)
{
    const Tile tl = a.tiles[t];
    const DevReplica r = a.reps[tl.rep];
    for (int k = 0; k < 3; ++k) f.L[k] = r.L[k];
    grid_shift(r, step, f.S);
    f.base = r.cell_base;
    f.beg = tl.begin;
    f.end = tl.end;
}

template <typename Real, bool PRE>
__global__ void __launch_bounds__(256) k_ang_sums(StepArgs a, void *words)
{
    typedef typename AngWord<Real>::type W;
    __shared__ TileFrame sf;
    W *w = reinterpret_cast<W *>(words);
    const int64_t C = a.n_cells;
    const int64_t step = *a.d_step;
    const Real m = solvent_mass<Real>(a);
    const Real *X = reinterpret_cast<const Real *>(a.x), *Y = reinterpret_cast<const Real *>(a.y);
    const Real *Z = reinterpret_cast<const Real *>(a.z), *VX = reinterpret_cast<const Real *>(a.vx);
    const Real *VY = reinterpret_cast<const Real *>(a.vy), *VZ = reinterpret_cast<const Real *>(a.vz);
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) load_frame(a, t, step, sf);
        __syncthreads();
        const TileFrame f = sf;
        for (int64_t i = f.beg + threadIdx.x; i < f.end; i += blockDim.x) {
            const Real r[3] = {X[i], Y[i], Z[i]};
            const Real v[3] = {VX[i], VY[i], VZ[i]};
            int Q[3], cc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int Xk = lattice_X(r[k]);
                cc[k] = axis_cell(Xk, f.S[k], f.L[k]);
                Q[k] = (Xk - f.S[k]) & 0xFFFFF;
            }
            const int64_t c = f.base + cc[0] + (int64_t)f.L[0] * (cc[1] + (int64_t)f.L[1] * cc[2]);
            const W P[3] = {mom_term(m, v[0]), mom_term(m, v[1]), mom_term(m, v[2])};
            const W q[3] = {(W)Q[0], (W)Q[1], (W)Q[2]};
            const W L[3] = {q[1] * P[2] - q[2] * P[1], q[2] * P[0] - q[0] * P[2], q[0] * P[1] - q[1] * P[0]};
            if (PRE) {
                ang_red(w + 0 * C + c, (W)1);
#pragma unroll
                for (int k = 0; k < 3; ++k) ang_red(w + (1 + k) * C + c, q[k]);
                ang_red(w + 4 * C + c, q[0] * q[0]);
                ang_red(w + 5 * C + c, q[1] * q[1]);
                ang_red(w + 6 * C + c, q[2] * q[2]);
                ang_red(w + 7 * C + c, q[0] * q[1]);
                ang_red(w + 8 * C + c, q[0] * q[2]);
                ang_red(w + 9 * C + c, q[1] * q[2]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ang_red(w + (10 + k) * C + c, L[k]);
                    ang_red(w + (13 + k) * C + c, P[k]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ang_red(w + (10 + k) * C + c, -L[k]);
                    ang_red(w + (13 + k) * C + c, -P[k]);
                }
            }
        }
    }
}

// per-cell record of the correction: sum Q, N and w' = w / (N 2^20)
template <typename Real> struct AngParams;
template <> struct AngParams<float> { uint32_t sq[3]; int32_t n; float w[3]; float pad; };
template <> struct AngParams<double> { double sq[3]; double n; double w[3]; double pad; };
static_assert(sizeof(AngParams<float>) == 32 && sizeof(AngParams<double>) == 64, "record sizes");

// w from the words of one cell (lattice units: Q in 2^-20, P in pscale)
template <typename W>
__device__ void cell_omega(const W (&wd)[ANG_WORDS], double m, double pscale, double om[3])
{
    om[0] = om[1] = om[2] = 0.0;
    const double N = (double)wd[0];
    if (N < 2.0) return;
    const double sQ[3] = {(double)wd[1], (double)wd[2], (double)wd[3]};
    const double Qc[3] = {sQ[0] / N, sQ[1] / N, sQ[2] / N};
    // lattice covariance C (exact sums; one rounding in the centre term)
    double Cm[3][3];
    Cm[0][0] = (double)wd[4] - sQ[0] * sQ[0] / N;
    Cm[1][1] = (double)wd[5] - sQ[1] * sQ[1] / N;
    Cm[2][2] = (double)wd[6] - sQ[2] * sQ[2] / N;
    Cm[0][1] = Cm[1][0] = (double)wd[7] - sQ[0] * sQ[1] / N;
    Cm[0][2] = Cm[2][0] = (double)wd[8] - sQ[0] * sQ[2] / N;
    Cm[1][2] = Cm[2][1] = (double)wd[9] - sQ[1] * sQ[2] / N;
    const double tr = Cm[0][0] + Cm[1][1] + Cm[2][2];
    // angular-momentum change about the centre, in units of 2^-20 pscale
    const double dP[3] = {(double)wd[13], (double)wd[14], (double)wd[15]};
    double dL[3] = {(double)wd[10] - (Qc[1] * dP[2] - Qc[2] * dP[1]),
                    (double)wd[11] - (Qc[2] * dP[0] - Qc[0] * dP[2]),
                    (double)wd[12] - (Qc[0] * dP[1] - Qc[1] * dP[0])};
    if (!(tr > 0.0)) return;                  // every member on one lattice point
    // G = tr(C) I - C = Pi / (m 2^-40); solve G x = dL
    double G[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[i][j] = (i == j ? tr : 0.0) - Cm[i][j];
    const double tol = 1e-12 * tr;
    double x[3];
    bool ok = G[0][0] > tol;
    double l00 = 0, l10 = 0, l20 = 0, l11 = 0, l21 = 0, l22 = 0;
    if (ok) {
        l00 = sqrt(G[0][0]);
        l10 = G[1][0] / l00;
        l20 = G[2][0] / l00;
        const double d1 = G[1][1] - l10 * l10;
        ok = d1 > tol;
        if (ok) {
            l11 = sqrt(d1);
            l21 = (G[2][1] - l20 * l10) / l11;
            const double d2 = G[2][2] - l20 * l20 - l21 * l21;
            ok = d2 > tol;
            if (ok) l22 = sqrt(d2);
        }
    }
    if (ok) {
        const double y0 = dL[0] / l00;
        const double y1 = (dL[1] - l10 * y0) / l11;
        const double y2 = (dL[2] - l20 * y0 - l21 * y1) / l22;
        x[2] = y2 / l22;
        x[1] = (y1 - l21 * x[2]) / l11;
        x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    } else {
        // collinear members: C = tr(C) d d^T, G = tr(C) (I - d d^T); least-norm x
        // = (dL - d (d.dL)) / tr(C) with d d^T = C / tr(C)
        for (int i = 0; i < 3; ++i) {
            const double CdL = Cm[i][0] * dL[0] + Cm[i][1] * dL[1] + Cm[i][2] * dL[2];
            x[i] = (dL[i] - CdL / tr) / tr;
        }
    }
    // Pi w = dL_phys: Pi = m 2^-40 G, dL_phys = 2^-20 pscale dL
    const double s = pscale * 1048576.0 / m;
    for (int k = 0; k < 3; ++k) om[k] = x[k] * s;
}

template <typename Real>
__global__ void __launch_bounds__(256) k_ang_params(StepArgs a, void *words, AngParams<Real> *params)
{
    typedef typename AngWord<Real>::type W;
    W *w = reinterpret_cast<W *>(words);
    const int64_t C = a.n_cells;
    const double m = sizeof(Real) == 4 ? (double)a.m_solvent_f : a.m_solvent;   // the mass of the P terms
    const double pscale = sizeof(Real) == 4 ? 0x1p-20 : 1.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        W wd[ANG_WORDS];
#pragma unroll
        for (int k = 0; k < ANG_WORDS; ++k) {
            wd[k] = w[k * C + c];
            w[k * C + c] = (W)0;
        }
        double om[3];
        cell_omega(wd, m, pscale, om);
        const double n = (double)wd[0];
        const double s = n >= 2.0 ? 1.0 / (n * 1048576.0) : 0.0;
        AngParams<Real> o;
        for (int k = 0; k < 3; ++k) {
            o.sq[k] = (decltype(o.sq[0]))wd[1 + k];
            o.w[k] = (Real)(om[k] * s);
        }
        o.n = (decltype(o.n))wd[0];
        o.pad = (Real)0;
        params[c] = o;
    }
}

// exact integer offset N Q - sum Q (|.| < N 2^20) in the working precision
__device__ __forceinline__ float offset_real(const AngParams<float> &p, int Q, int k)
{
    return ll2f((long long)p.n * Q - (long long)p.sq[k]);
}
__device__ __forceinline__ double offset_real(const AngParams<double> &p, int Q, int k)
{
    return p.n * (double)Q - p.sq[k];   // integers below 2^53: exact
}

template <typename Real>
__global__ void __launch_bounds__(256) k_ang_apply(StepArgs a, const AngParams<Real> *params)
{
    __shared__ TileFrame sf;
    const int64_t step = *a.d_step;
    const Real *X = reinterpret_cast<const Real *>(a.x), *Y = reinterpret_cast<const Real *>(a.y);
    const Real *Z = reinterpret_cast<const Real *>(a.z);
    Real *VX = reinterpret_cast<Real *>(a.vx), *VY = reinterpret_cast<Real *>(a.vy);
    Real *VZ = reinterpret_cast<Real *>(a.vz);
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) load_frame(a, t, step, sf);
        __syncthreads();
        const TileFrame f = sf;
        for (int64_t i = f.beg + threadIdx.x; i < f.end; i += blockDim.x) {
            const Real r[3] = {X[i], Y[i], Z[i]};
            int cc[3], Q[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int Xk = lattice_X(r[k]);
                cc[k] = axis_cell(Xk, f.S[k], f.L[k]);
                Q[k] = (Xk - f.S[k]) & 0xFFFFF;
            }
            const int64_t c = f.base + cc[0] + (int64_t)f.L[0] * (cc[1] + (int64_t)f.L[1] * cc[2]);
            const AngParams<Real> p = params[c];
            const Real rc[3] = {offset_real(p, Q[0], 0), offset_real(p, Q[1], 1), offset_real(p, Q[2], 2)};
            const Real wx = p.w[0], wy = p.w[1], wz = p.w[2];
            VX[i] = VX[i] + (wy * rc[2] - wz * rc[1]);
            VY[i] = VY[i] + (wz * rc[0] - wx * rc[2]);
            VZ[i] = VZ[i] + (wx * rc[1] - wy * rc[0]);
        }
    }
}

}  // namespace

size_t angular_param_bytes(int precision)
{
    return precision == 1 ? sizeof(AngParams<float>) : sizeof(AngParams<double>);
}

void launch_angular(const StepArgs &a, int phase, void *words, void *params, int num_sms, cudaStream_t s)
{
    if (a.n_cells == 0) return;
    const int grid_p = std::max(1, num_sms * 16);
    const int grid_t = (int)std::max(1, std::min(a.n_tiles, num_sms * 16));
    const bool p32 = a.precision == 1;
    switch (phase) {
    case ANG_PRE:
        if (a.n_tiles == 0) return;
        if (p32) k_ang_sums<float, true><<<grid_t, 256, 0, s>>>(a, words);
        else k_ang_sums<double, true><<<grid_t, 256, 0, s>>>(a, words);
        break;
    case ANG_POST:
        if (a.n_tiles == 0) return;
        if (p32) k_ang_sums<float, false><<<grid_t, 256, 0, s>>>(a, words);
        else k_ang_sums<double, false><<<grid_t, 256, 0, s>>>(a, words);
        break;
    case ANG_PARAMS:
        if (p32) k_ang_params<float><<<grid_p, 256, 0, s>>>(a, words, reinterpret_cast<AngParams<float> *>(params));
        else k_ang_params<double><<<grid_p, 256, 0, s>>>(a, words, reinterpret_cast<AngParams<double> *>(params));
        break;
    case ANG_APPLY:
        if (a.n_tiles == 0) return;
        if (p32) k_ang_apply<float><<<grid_t, 256, 0, s>>>(a, reinterpret_cast<const AngParams<float> *>(params));
        else k_ang_apply<double><<<grid_t, 256, 0, s>>>(a, reinterpret_cast<const AngParams<double> *>(params));
        break;
    default:
        break;
    }
}

}  // namespace mpcd
