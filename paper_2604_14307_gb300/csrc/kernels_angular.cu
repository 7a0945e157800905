// Angular-momentum-conserving variants of the collision rules (SRD+a and
// MPCD-AT+a: the modification of the rules that Sec. II.A of arXiv 2604.14307
// cites from Noguchi and Gompper): the solvent's passes and the per-cell solve;
// the colloid sites' share lives beside the other site kernels.
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
//   k_ang_shift       the grid shift of every replica (once per collision)
//   k_ang_sums<PRE>   solvent, before the rule: count, sum Q, sum Q_a Q_b,
//                     + sum Q x P, + sum P (the sites add theirs from the
//                     thermalised velocities, kernels_bodies.cu)
//   k_ang_sums<POST>  after the rule: - sum Q x P*, - sum P* (sites likewise)
//   k_ang_params      per cell: centre of mass, Pi and the angular-momentum
//                     change in FP64, w by the adjugate of Pi (least-norm form
//                     for collinear members); clears the words
//   k_ang_apply       solvent: v = v* + w' x (M Q - sum mu Q), w' = w / (M 2^20);
//                     the site POST coupling applies the same to the sites
//                     before it transfers their momentum change to the body
// Word layout and record: AW_* and AngParams in mpcd_internal.cuh.  The
// geometric sums are kept per species (solvent, sites) and exact; masses enter
// in the per-cell solve (P32: mu = round(m 2^24), the quantised masses of the
// cell words).  The offset from the centre is formed as the exact integer
// M Q - sum mu Q: for nearly collinear members w is large along their line
// while the offsets across it are small, and an offset rounded in the working
// precision would carry an error of order eps |w| into the velocity.
// P32: every word an int64 sum (exact and independent of the order of the
// atomics; wrap-around of partial sums cancels as long as the final sum lies
// within +-2^63).  P64: the Q sums are exact integers in double, the momentum
// sums FP64 atomics.
#include <algorithm>

#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

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

// per-replica grid shift of the collision, computed once per collision
__global__ void k_ang_shift(StepArgs a, int4 *shifts)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_rep) return;
    int32_t S[3];
    grid_shift(a.reps[r], *a.d_step, S);
    shifts[r] = make_int4(S[0], S[1], S[2], 0);
}

__device__ __forceinline__ void ld4v(const float *p, float (&o)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4v(const double *p, double (&o)[4])
{
    const double2 t0 = reinterpret_cast<const double2 *>(p)[0], t1 = reinterpret_cast<const double2 *>(p)[1];
    o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}
__device__ __forceinline__ void st4v(float *p, const float (&o)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4v(double *p, const double (&o)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
}

// cell and lattice offset Q of each of a thread's 4 particles
template <typename Real>
__device__ __forceinline__ void cells4(const Real (&x)[4], const Real (&y)[4], const Real (&z)[4], int4 S,
                                       const DevReplica &r, int64_t (&c)[4], int (&Q)[4][3])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int X[3] = {lattice_X(x[j]), lattice_X(y[j]), lattice_X(z[j])};
        const int Sk[3] = {S.x, S.y, S.z};
        int cc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cc[k] = axis_cell(X[k], Sk[k], r.L[k]);
            Q[j][k] = (X[k] - Sk[k]) & 0xFFFFF;
        }
        c[j] = r.cell_base + cc[0] + (int64_t)r.L[0] * (cc[1] + (int64_t)r.L[1] * cc[2]);
    }
}

// One warp per tile; each lane takes 4 consecutive particles (128-bit loads;
// tiles start on multiples of 8 slots, and the slots past a replica's last
// particle are allocated padding), merges runs of equal cells in registers and
// issues one atomic per word and run.  PRE adds the solvent's 16 terms, POST
// subtracts the rule's new momentum terms.
template <typename Real, bool PRE>
__global__ void __launch_bounds__(256) k_ang_sums(StepArgs a)
{
    typedef typename AngWord<Real>::type W;
    W *w = reinterpret_cast<W *>(a.ang_words);
    const int4 *shifts = a.ang_shift;
    const int64_t C = a.n_cells;
    const Real m = solvent_mass<Real>(a);
    const Real *X = reinterpret_cast<const Real *>(a.x), *Y = reinterpret_cast<const Real *>(a.y);
    const Real *Z = reinterpret_cast<const Real *>(a.z), *VX = reinterpret_cast<const Real *>(a.vx);
    const Real *VY = reinterpret_cast<const Real *>(a.vy), *VZ = reinterpret_cast<const Real *>(a.vz);
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < a.n_tiles; t += gridDim.x * warps) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        const int4 S = shifts[tl.rep];
        for (int64_t i = tl.begin + 4 * lane; i < tl.end; i += 128) {
            const int nv = (int)min((int64_t)4, tl.end - i);
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            ld4v(X + i, x); ld4v(Y + i, y); ld4v(Z + i, z);
            ld4v(VX + i, vx); ld4v(VY + i, vy); ld4v(VZ + i, vz);
            int64_t c[4];
            int Q[4][3];
            cells4(x, y, z, S, r, c, Q);
            W P[4][3];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                P[j][0] = mom_term(m, vx[j]); P[j][1] = mom_term(m, vy[j]); P[j][2] = mom_term(m, vz[j]);
            }
            bool join[4], head[4];   // join[j]: particle j+1 is in j's cell
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                join[j] = j + 1 < nv && c[j + 1] == c[j];
                head[j] = j < nv && (j == 0 || c[j] != c[j - 1]);
            }
            // the solvent's words: count, sum Q, sum Q_a Q_b (PRE only), then
            // the momentum words; k indexes the 16 terms, wk the word
#pragma unroll
            for (int k = PRE ? 0 : 10; k < 16; ++k) {
                const int wk = k == 0 ? AW_COUNT : k < 4 ? AW_SQ + k - 1 : k < 10 ? AW_QQ + k - 4
                                                        : k < 13 ? AW_L + k - 10 : AW_P + k - 13;
                W v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const W q0 = (W)Q[j][0], q1 = (W)Q[j][1], q2 = (W)Q[j][2];
                    W e;
                    switch (k) {
                    case 0: e = (W)1; break;
                    case 1: e = q0; break;
                    case 2: e = q1; break;
                    case 3: e = q2; break;
                    case 4: e = q0 * q0; break;
                    case 5: e = q1 * q1; break;
                    case 6: e = q2 * q2; break;
                    case 7: e = q0 * q1; break;
                    case 8: e = q0 * q2; break;
                    case 9: e = q1 * q2; break;
                    case 10: e = q1 * P[j][2] - q2 * P[j][1]; break;
                    case 11: e = q2 * P[j][0] - q0 * P[j][2]; break;
                    case 12: e = q0 * P[j][1] - q1 * P[j][0]; break;
                    default: e = P[j][k - 13]; break;
                    }
                    v[j] = PRE ? e : -e;
                }
#pragma unroll
                for (int j = 2; j >= 0; --j)
                    if (join[j]) v[j] += v[j + 1];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (head[j]) ang_red(w + wk * C + c[j], v[j]);
            }
        }
    }
}

// record of one cell from its words.  mu_s, mu_b: the solvent and site mass
// in the units of the form (P32: round(m 2^24), P64: m); pscale: the unit of
// the P terms (P32: 2^-20, P64: 1); mscale: the unit of mu (P32: 2^-24, P64: 1).
template <typename Real, typename W>
__device__ void cell_record(const W (&wd)[ANG_WORDS], double mu_s, double mu_b, double pscale, double mscale,
                            AngParams<Real> &o)
{
    const long long cnt = (long long)wd[AW_COUNT];
    const double ns = (double)(cnt & 0xFFF), nb = (double)((cnt >> 12) & 0x3FF);
    const double M = ns * mu_s + nb * mu_b;     // exact (integers below 2^53 in P32)
    double sw[3];
    for (int k = 0; k < 3; ++k) {
        if constexpr (sizeof(Real) == 4) {
            // exact in int64: mu Q sums below M 2^20
            const long long v = (long long)mu_s * (long long)wd[AW_SQ + k] + (long long)mu_b * (long long)wd[AW_SQB + k];
            o.sw[k] = v;
            sw[k] = (double)v;
        } else {
            sw[k] = mu_s * (double)wd[AW_SQ + k] + mu_b * (double)wd[AW_SQB + k];
            o.sw[k] = sw[k];
        }
        o.w[k] = (Real)0;
    }
    if constexpr (sizeof(Real) == 4) o.M = (long long)M;
    else o.M = M;
    o.pad = (Real)0;
    if (ns + nb < 2.0) return;
    const double iM = 1.0 / M;
    const double Qc[3] = {sw[0] * iM, sw[1] * iM, sw[2] * iM};
    // mass-weighted lattice covariance about the centre of mass
    double Cm[3][3];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
        const double v = mu_s * (double)wd[AW_QQ + q] + mu_b * (double)wd[AW_QQB + q] - sw[ia[q]] * Qc[ib[q]];
        Cm[ia[q]][ib[q]] = Cm[ib[q]][ia[q]] = v;
    }
    const double tr = Cm[0][0] + Cm[1][1] + Cm[2][2];
    if (!(tr > 0.0)) return;                  // every member on one lattice point
    // angular-momentum change about the centre (units 2^-20 pscale)
    const double dP[3] = {(double)wd[AW_P], (double)wd[AW_P + 1], (double)wd[AW_P + 2]};
    const double dL[3] = {(double)wd[AW_L] - (Qc[1] * dP[2] - Qc[2] * dP[1]),
                          (double)wd[AW_L + 1] - (Qc[2] * dP[0] - Qc[0] * dP[2]),
                          (double)wd[AW_L + 2] - (Qc[0] * dP[1] - Qc[1] * dP[0])};
    // G = tr(C) I - C = Pi / (mscale 2^-40); solve G x = dL by its adjugate
    const double a00 = tr - Cm[0][0], a11 = tr - Cm[1][1], a22 = tr - Cm[2][2];
    const double a01 = -Cm[0][1], a02 = -Cm[0][2], a12 = -Cm[1][2];
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    double x[3];
    if (det > 1e-12 * tr * tr * tr) {
        const double inv = 1.0 / det;
        x[0] = (c00 * dL[0] + c01 * dL[1] + c02 * dL[2]) * inv;
        x[1] = (c01 * dL[0] + c11 * dL[1] + c12 * dL[2]) * inv;
        x[2] = (c02 * dL[0] + c12 * dL[1] + c22 * dL[2]) * inv;
    } else {
        // collinear members: C = tr(C) d d^T, G = tr(C) (I - d d^T); least-norm x
        // = (dL - d (d.dL)) / tr(C) with d d^T = C / tr(C)
        const double it = 1.0 / tr;
        for (int i = 0; i < 3; ++i) {
            const double CdL = Cm[i][0] * dL[0] + Cm[i][1] * dL[1] + Cm[i][2] * dL[2];
            x[i] = (dL[i] - CdL * it) * it;
        }
    }
    // Pi w = dL_phys with Pi = mscale 2^-40 G and dL_phys = 2^-20 pscale dL;
    // the record keeps w' = w / (M 2^20)
    const double s = pscale / (mscale * M);
    for (int k = 0; k < 3; ++k) o.w[k] = (Real)(x[k] * s);
}

template <typename Real>
__global__ void __launch_bounds__(256) k_ang_params(StepArgs a)
{
    typedef typename AngWord<Real>::type W;
    W *w = reinterpret_cast<W *>(a.ang_words);
    AngParams<Real> *params = reinterpret_cast<AngParams<Real> *>(const_cast<void *>(a.ang_params));
    const int64_t C = a.n_cells;
    const bool p32 = sizeof(Real) == 4;
    const double mu_s = p32 ? (double)a.qm_solvent : a.m_solvent;
    const double mu_b = p32 ? (double)a.qm_site : a.m_site;
    const double pscale = p32 ? 0x1p-20 : 1.0, mscale = p32 ? 0x1p-24 : 1.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        W wd[ANG_WORDS];
#pragma unroll
        for (int k = 0; k < ANG_WORDS; ++k) {
            wd[k] = w[k * C + c];
            w[k * C + c] = (W)0;
        }
        AngParams<Real> o;
        cell_record<Real>(wd, mu_s, mu_b, pscale, mscale, o);
        params[c] = o;
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_ang_apply(StepArgs a)
{
    const AngParams<Real> *params = reinterpret_cast<const AngParams<Real> *>(a.ang_params);
    const int4 *shifts = a.ang_shift;
    const Real *X = reinterpret_cast<const Real *>(a.x), *Y = reinterpret_cast<const Real *>(a.y);
    const Real *Z = reinterpret_cast<const Real *>(a.z);
    Real *VX = reinterpret_cast<Real *>(a.vx), *VY = reinterpret_cast<Real *>(a.vy);
    Real *VZ = reinterpret_cast<Real *>(a.vz);
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < a.n_tiles; t += gridDim.x * warps) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        const int4 S = shifts[tl.rep];
        for (int64_t i = tl.begin + 4 * lane; i < tl.end; i += 128) {
            const int nv = (int)min((int64_t)4, tl.end - i);
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            ld4v(X + i, x); ld4v(Y + i, y); ld4v(Z + i, z);
            ld4v(VX + i, vx); ld4v(VY + i, vy); ld4v(VZ + i, vz);
            int64_t c[4];
            int Q[4][3];
            cells4(x, y, z, S, r, c, Q);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nv) break;
                Real v[3] = {vx[j], vy[j], vz[j]};
                ang_correct(params[c[j]], Q[j], v);
                vx[j] = v[0]; vy[j] = v[1]; vz[j] = v[2];
            }
            if (nv == 4) {
                st4v(VX + i, vx); st4v(VY + i, vy); st4v(VZ + i, vz);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nv) { VX[i + j] = vx[j]; VY[i + j] = vy[j]; VZ[i + j] = vz[j]; }
            }
        }
    }
}

}  // namespace

size_t angular_param_bytes(int precision)
{
    static_assert(sizeof(AngParams<float>) == 48 && sizeof(AngParams<double>) == 64, "record sizes");
    return precision == 1 ? sizeof(AngParams<float>) : sizeof(AngParams<double>);
}

void launch_angular(const StepArgs &a, int phase, int num_sms, cudaStream_t s)
{
    if (a.n_cells == 0) return;
    const int grid_p = std::max(1, num_sms * 16);
    const int grid_t = (int)std::max(1, std::min((a.n_tiles + 7) / 8, num_sms * 8));   // 8 warps, one tile each
    const bool p32 = a.precision == 1;
    switch (phase) {
    case ANG_PRE:
        k_ang_shift<<<(a.n_rep + 127) / 128, 128, 0, s>>>(a, a.ang_shift);
        if (a.n_tiles == 0) return;
        if (p32) k_ang_sums<float, true><<<grid_t, 256, 0, s>>>(a);
        else k_ang_sums<double, true><<<grid_t, 256, 0, s>>>(a);
        break;
    case ANG_POST:
        if (a.n_tiles == 0) return;
        if (p32) k_ang_sums<float, false><<<grid_t, 256, 0, s>>>(a);
        else k_ang_sums<double, false><<<grid_t, 256, 0, s>>>(a);
        break;
    case ANG_PARAMS:
        if (p32) k_ang_params<float><<<grid_p, 256, 0, s>>>(a);
        else k_ang_params<double><<<grid_p, 256, 0, s>>>(a);
        break;
    case ANG_APPLY:
        if (a.n_tiles == 0) return;
        if (p32) k_ang_apply<float><<<grid_t, 256, 0, s>>>(a);
        else k_ang_apply<double><<<grid_t, 256, 0, s>>>(a);
        break;
    default:
        break;
    }
}

}  // namespace mpcd
