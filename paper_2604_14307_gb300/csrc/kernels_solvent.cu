// Solvent and cell kernels of the MPCD step (Sec. II.A of arXiv 2604.14307).
//
// k_solvent   one pass over the solvent that, depending on FLAGS, applies the
//             collision of the current step (SRD rotation by alpha about the
//             cell axis with thermostat scale kappa, or the MPCD-AT rule),
//             streams ballistically with periodic wrap, and bins the streamed
//             particle into the cell sums of the next collision (random grid
//             shift, Sec. II.A).  Fused (all three flags) it reads and writes
//             r and v once per step: 48 B per particle in FP32.
//             Each thread owns 4 consecutive particles loaded with 128-bit SoA
//             loads (cache-streaming hints keep the cell arrays in L2); runs
//             of equal cells are merged in registers before the atomics.
// k_params    per cell: sums -> centre-of-mass velocity u, SRD axis, thermostat
//             scale (Huang et al.; Eq. 6 with n = 3(Nc-1)) or AT mean noise;
//             clears the sums for the next collision.
// re-sort     counting sort of the solvent by cell (histogram, scan, scatter,
//             optional per-cell order by tag) for memory locality; it changes
//             no result.
// The solvent pass has four launch forms that give bit-identical results:
// direct loads (k_solvent), a CTA-wide three-stage bulk-copy ring
// (k_solvent_staged), a warp-specialised three-stage ring (k_solvent_ws) and a
// three-stage ring per warp (k_solvent_wt).  Streaming takes an optional
// constant force (the balancing force of the sedimentation protocol).
// Transport protocols of Sec. III.B: the reverse non-equilibrium exchange
// (k_rnemd_scan, k_rnemd_filter, k_rnemd_select) and the velocity profile.
#include <map>
#include <mutex>
#include <utility>

#include "mpcd_internal.cuh"

namespace mpcd {

// ------------------------------------------------------------------ helpers
// (x + 1/2) 2^-32 from all 32 bits, relative error <= 2^-24 (never 0; 1 only
// when x rounds up to 2^32)
__device__ __forceinline__ float u01f(uint32_t x)
{
    return __fmaf_rn(__uint2float_rn(x), 2.3283064365386962890625e-10f, 1.16415321826934814453125e-10f);
}
__device__ __forceinline__ double u01d(uint32_t x)
{
    return ((double)x + 0.5) * 2.3283064365386962890625e-10;     // (x + 1/2) 2^-32
}

// -2 ln u for u = (x + 1/2) 2^-32 with full relative precision also near u = 1,
// where 1 - u = (~x + 1/2) 2^-32 is formed exactly from the integer complement
__device__ __forceinline__ float neg2log(uint32_t x)
{
    return (x & 0x80000000u) ? -2.0f * log1pf(-u01f(~x)) : -2.0f * __logf(u01f(x));
}

// three standard normals from one Philox block (Box-Muller); the angles are
// shifted by pi into [-pi, pi) where the fast sine/cosine are accurate
__device__ __forceinline__ void normals3(uint4 w, float n[3])
{
    const float r1 = sqrtf(neg2log(w.x));
    const float r2 = sqrtf(neg2log(w.z));
    float s1, c1;
    __sincosf(6.283185307179586f * (u01f(w.y) - 0.5f), &s1, &c1);
    n[0] = -r1 * c1;
    n[1] = -r1 * s1;
    n[2] = -r2 * __cosf(6.283185307179586f * (u01f(w.w) - 0.5f));
}
__device__ __forceinline__ void normals3(uint4 w, double n[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = sqrt(-2.0 * log(u01d(w.x)));
    double r2 = sqrt(-2.0 * log(u01d(w.z)));
    double s1, c1;
    sincos(two_pi * u01d(w.y), &s1, &c1);
    n[0] = r1 * c1;
    n[1] = r1 * s1;
    n[2] = r2 * cos(two_pi * u01d(w.w));
}

// binning rule: X = floor(x 2^20), cell = floor((X - S) / 2^20) mod L
__device__ __forceinline__ int cell_axis(float x, int S, int L)
{
    int c = (__float2int_rd(x * 1048576.0f) - S) >> 20;
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    return ((unsigned)c < (unsigned)L) ? c : 0;   // only a non-finite position gets here; it is flagged

}
__device__ __forceinline__ int cell_axis(double x, int S, int L)
{
    int c = (__double2int_rd(x * 1048576.0) - S) >> 20;
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    return ((unsigned)c < (unsigned)L) ? c : 0;   // only a non-finite position gets here; it is flagged

}
// The same rule in float32 without a conversion instruction (the solvent
// passes).  With S an integer, floor((floor(x 2^20) - S) / 2^20) =
// floor(x - s) for s = S 2^-20, which float32 holds exactly.  x - s rounded
// toward -inf has the floor of the exact difference (the rounding is monotone
// and keeps integers), and floor_magic reads that floor off the mantissa
// (|x - s| < 2^11 here).
// For x in [0, L) and |s| <= 1/2 the floor lies in [-1, L]: the top is wrapped
// by one select and -1 by an unsigned minimum with L - 1, which also keeps a
// non-finite position's cell inside the box (such a position is flagged).
__device__ __forceinline__ int cell_axis_f(float x, float s, int L)
{
    int c = floor_magic_int(floor_magic(__fsub_rd(x, s)));
    c = c == L ? 0 : c;
    return (int)min((unsigned)c, (unsigned)(L - 1));
}
// grid shift of one axis in the form the binning of a precision takes
template <typename Real> struct ShiftT { typedef int32_t type; };
template <> struct ShiftT<float> { typedef float type; };
__device__ __forceinline__ int32_t shift_as(int32_t S, int32_t) { return S; }
__device__ __forceinline__ float shift_as(int32_t S, float)
{
    return __fmul_rn(__int2float_rn(S), 9.5367431640625e-07f);   // S 2^-20, exact for |S| <= 2^19
}
__device__ __forceinline__ int cell_bin(float x, float s, int L) { return cell_axis_f(x, s, L); }
__device__ __forceinline__ int cell_bin(double x, int32_t S, int L) { return cell_axis(x, S, L); }

// streaming x + v dt with periodic wrap, unfused (same rounding as the oracle)
__device__ __forceinline__ float drift(float x, float v, float dt, float L, int &bad)
{
    float y = __fadd_rn(x, __fmul_rn(v, dt));
    if (y >= L) y = __fsub_rn(y, L);
    else if (y < 0.0f) { y = __fadd_rn(y, L); if (y >= L) y = 0.0f; }
    bad |= !(y >= 0.0f && y < L);
    return y;
}
__device__ __forceinline__ double drift(double x, double v, double dt, double L, int &bad)
{
    double y = __dadd_rn(x, __dmul_rn(v, dt));
    if (y >= L) y = __dsub_rn(y, L);
    else if (y < 0.0) { y = __dadd_rn(y, L); if (y >= L) y = 0.0; }
    bad |= !(y >= 0.0 && y < L);
    return y;
}
// Streaming under a constant force (the solvent's share of the balancing
// force of the sedimentation protocol): v += a dt/2, x += v dt, v += a dt/2,
// exact for a constant force; with no force the plain drift.
__device__ __forceinline__ float kick(float v, float h) { return __fadd_rn(v, h); }
__device__ __forceinline__ double kick(double v, double h) { return __dadd_rn(v, h); }


__device__ __forceinline__ void ld4(const float *p, float (&o)[4])
{
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4])
{
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&o)[4])
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(o[0], o[1], o[2], o[3]));
}
__device__ __forceinline__ void st4(double *p, const double (&o)[4])
{
    __stcs(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
    __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(o[2], o[3]));
}

// collision parameters of one cell
template <typename Real> struct CellParams { Real ux, uy, uz, kappa, ax, ay, az; };

__device__ __forceinline__ CellParams<float> load_params(const void *params, int64_t c)
{
    const float4 *p = reinterpret_cast<const float4 *>(params) + 2 * c;
    float4 a = p[0], b = p[1];
    return {a.x, a.y, a.z, a.w, b.x, b.y, b.z};
}
__device__ __forceinline__ CellParams<double> load_params_d(const void *params, int64_t c)
{
    const double2 *p = reinterpret_cast<const double2 *>(params) + 4 * c;
    double2 a = p[0], b = p[1], d = p[2], e = p[3];
    return {a.x, a.y, b.x, b.y, d.x, d.y, e.x};
}
template <typename Real> __device__ __forceinline__ CellParams<Real> get_params(const void *pr, int64_t c);
template <> __device__ __forceinline__ CellParams<float> get_params<float>(const void *pr, int64_t c)
{
    return load_params(pr, c);
}
template <> __device__ __forceinline__ CellParams<double> get_params<double>(const void *pr, int64_t c)
{
    return load_params_d(pr, c);
}

template <typename Real> struct Consts;
template <> struct Consts<float> {
    __device__ static float kT(const StepArgs &a) { return a.kTf; }
    __device__ static float dt(const StepArgs &a) { return a.dtf; }
    __device__ static float m(const StepArgs &a) { return a.m_solvent_f; }
    __device__ static float ca(const StepArgs &a) { return a.cos_af; }
    __device__ static float sa(const StepArgs &a) { return a.sin_af; }
    __device__ static float ah(const StepArgs &a, int k) { return a.ahf[k]; }
};
template <> struct Consts<double> {
    __device__ static double kT(const StepArgs &a) { return a.kT; }
    __device__ static double dt(const StepArgs &a) { return a.dt; }
    __device__ static double m(const StepArgs &a) { return a.m_solvent; }
    __device__ static double ca(const StepArgs &a) { return a.cos_a; }
    __device__ static double sa(const StepArgs &a) { return a.sin_a; }
    __device__ static double ah(const StepArgs &a, int k) { return a.ah[k]; }
};

// SRD: v' = u + kappa R(n, alpha)(v - u)  (Rodrigues)
template <typename Real>
__device__ __forceinline__ void srd_rotate(const CellParams<Real> &p, Real ca, Real sa, Real &vx,
                                           Real &vy, Real &vz)
{
    Real wx = vx - p.ux, wy = vy - p.uy, wz = vz - p.uz;
    Real nd = p.ax * wx + p.ay * wy + p.az * wz;
    Real cx = p.ay * wz - p.az * wy, cy = p.az * wx - p.ax * wz, cz = p.ax * wy - p.ay * wx;
    Real t = nd * (Real(1) - ca);
    vx = p.ux + p.kappa * (wx * ca + cx * sa + p.ax * t);
    vy = p.uy + p.kappa * (wy * ca + cy * sa + p.ay * t);
    vz = p.uz + p.kappa * (wz * ca + cz * sa + p.az * t);
}

// word count of the cell sums
template <typename Real, int RULE> struct NWords;
template <> struct NWords<float, 0> { static constexpr int n = 3; };
template <> struct NWords<float, 1> { static constexpr int n = 4; };
template <> struct NWords<double, 0> { static constexpr int n = 6; };
template <> struct NWords<double, 1> { static constexpr int n = 8; };
template <typename Real> struct SumWord { typedef double type; };
template <> struct SumWord<float> { typedef long long type; };

// FP64 form: contributions of one particle (mass m, velocity v, AT noise xi)
// to the double sum arrays N, M, m v (3), m v.v (SRD) or m xi (3) (AT)
template <int RULE>
__device__ __forceinline__ void terms64(double m, double vx, double vy, double vz, const double *xi, double *w)
{
    w[0] = 1.0;
    w[1] = m;
    w[2] = m * vx;
    w[3] = m * vy;
    w[4] = m * vz;
    if (RULE == 0) {
        w[5] = m * (vx * vx + vy * vy + vz * vz);
    } else {
        w[5] = m * xi[0];
        w[6] = m * xi[1];
        w[7] = m * xi[2];
    }
}

__device__ __forceinline__ void red_add(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
__device__ __forceinline__ void red_add(double *p, double v) { atomicAdd(p, v); }

// Binning of a thread's 4 consecutive particles: cell under the shift S,
// per-particle fixed-point (P32) or double (P64) terms, runs of equal cells
// merged in registers, then one atomic per word and run.
template <typename Real, int RULE, bool COLLIDE, typename W, typename SH>
__device__ __forceinline__ void bin4(const StepArgs &a, const Real (&x)[4], const Real (&y)[4], const Real (&z)[4],
                                     const Real (&vx)[4], const Real (&vy)[4], const Real (&vz)[4],
                                     const uint32_t (&tg)[4], int nv, const SH *S, int L0, int L1, int L2,
                                     int base, const DevReplica &rr, int64_t step, Real m, Real sc, W *sums,
                                     int64_t C)
{
    int cc[4];
    Real xi[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cc[j] = base + cell_bin(x[j], S[0], L0) + L0 * (cell_bin(y[j], S[1], L1) + L1 * cell_bin(z[j], S[2], L2));
        xi[j][0] = xi[j][1] = xi[j][2] = Real(0);
        if (RULE == 1) {   // for every slot, so that the four draws interleave; runs past nv are dropped
            normals3(draw(rr, step + (COLLIDE ? 1 : 0), tg[j], TAG_AT, 0u), xi[j]);
            xi[j][0] *= sc; xi[j][1] *= sc; xi[j][2] *= sc;
        }
    }
    if constexpr (sizeof(Real) == 4) {
        // forward run merging: one running total, flushed when the cell changes
        constexpr int NW = Words32<RULE>::n;
        long long acc[MAX_WORDS32];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long w[MAX_WORDS32];
            record_terms<RULE>(m, vx[j], vy[j], vz[j], xi[j], false, w);
            if (j > 0 && j < nv && cc[j] == cc[j - 1]) {
#pragma unroll
                for (int k = 0; k < NW; ++k) acc[k] += w[k];
            } else {
                if (j > 0 && j - 1 < nv)
#pragma unroll
                    for (int k = 0; k < NW; ++k) red_add(sums + k * C + cc[j - 1], acc[k]);
#pragma unroll
                for (int k = 0; k < NW; ++k) acc[k] = w[k];
            }
        }
        if (nv == 4)
#pragma unroll
            for (int k = 0; k < NW; ++k) red_add(sums + k * C + cc[3], acc[k]);
    } else {
        constexpr int NW = RULE == 0 ? 6 : 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= nv) break;
            double w[NW];
            terms64<RULE>(m, vx[j], vy[j], vz[j], xi[j], w);
#pragma unroll
            for (int k = 0; k < NW; ++k) red_add(sums + k * C + cc[j], w[k]);
        }
    }
}

// --------------------------------------------------------------- the pass
template <typename Real, int RULE, int FLAGS>
__global__ void __launch_bounds__(512) k_solvent(StepArgs a)
{
    constexpr bool COLLIDE = FLAGS & SOLV_COLLIDE;
    constexpr bool STREAM = FLAGS & SOLV_STREAM;
    constexpr bool BIN = FLAGS & SOLV_BIN;
    typedef typename SumWord<Real>::type W;

    __shared__ int32_t sS[6];
    __shared__ typename ShiftT<Real>::type sF[6];   // sS in the binning's form
    __shared__ int32_t sL[3];
    __shared__ int32_t sbase;
    __shared__ int64_t sbeg, send;
    __shared__ uint32_t skey[2];

    const int64_t step = *a.d_step;
    const Real dt = Consts<Real>::dt(a), m = Consts<Real>::m(a), kT = Consts<Real>::kT(a);
    const Real ca = Consts<Real>::ca(a), sa = Consts<Real>::sa(a);
    const Real sc = sqrt(kT / m);
    Real *X = reinterpret_cast<Real *>(a.x), *Y = reinterpret_cast<Real *>(a.y);
    Real *Z = reinterpret_cast<Real *>(a.z), *VX = reinterpret_cast<Real *>(a.vx);
    Real *VY = reinterpret_cast<Real *>(a.vy), *VZ = reinterpret_cast<Real *>(a.vz);
    W *sums = reinterpret_cast<W *>(a.sums);
    const int64_t C = a.n_cells;
    int bad = 0;

    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            Tile tl = a.tiles[t];
            DevReplica r = a.reps[tl.rep];
            sL[0] = r.L[0]; sL[1] = r.L[1]; sL[2] = r.L[2];
            sbase = r.cell_base;
            sbeg = tl.begin;
            send = tl.end;
            skey[0] = r.key0;
            skey[1] = r.key1;
            if (COLLIDE) grid_shift(r, step, &sS[0]);
            if (BIN) grid_shift(r, step + (COLLIDE ? 1 : 0), &sS[3]);
            for (int c = 0; c < 6; ++c) sF[c] = shift_as(sS[c], typename ShiftT<Real>::type());
        }
        __syncthreads();
        const int L0 = sL[0], L1 = sL[1], L2 = sL[2], base = sbase;
        const Real Lx = (Real)L0, Ly = (Real)L1, Lz = (Real)L2;
        const int64_t beg = sbeg, end = send;
        DevReplica rr;
        rr.key0 = skey[0];
        rr.key1 = skey[1];

        for (int64_t i = beg + 4 * (int64_t)threadIdx.x; i < end; i += 4 * (int64_t)blockDim.x) {
            const int nv = (int)min((int64_t)4, end - i);
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            ld4(X + i, x); ld4(Y + i, y); ld4(Z + i, z);
            ld4(VX + i, vx); ld4(VY + i, vy); ld4(VZ + i, vz);
            uint32_t tg[4] = {0, 0, 0, 0};
            if (RULE == 1) {
                uint4 t4 = __ldcs(reinterpret_cast<const uint4 *>(a.tag + i));
                tg[0] = t4.x; tg[1] = t4.y; tg[2] = t4.z; tg[3] = t4.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nv) break;
                if (COLLIDE) {
                    int c = base + cell_bin(x[j], sF[0], L0) +
                            L0 * (cell_bin(y[j], sF[1], L1) + L1 * cell_bin(z[j], sF[2], L2));
                    CellParams<Real> p = get_params<Real>(a.params, c);
                    if (p.kappa >= Real(0)) {
                        if (RULE == 0) {
                            srd_rotate<Real>(p, ca, sa, vx[j], vy[j], vz[j]);
                        } else {
                            Real n[3];
                            normals3(draw(rr, step, tg[j], TAG_AT, 0u), n);
                            vx[j] = p.ux + sc * n[0] - p.ax;
                            vy[j] = p.uy + sc * n[1] - p.ay;
                            vz[j] = p.uz + sc * n[2] - p.az;
                        }
                    }
                }
                if (STREAM) {
                    if (a.accel) {
                        vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                        vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                        vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                    }
                    x[j] = drift(x[j], vx[j], dt, Lx, bad);
                    y[j] = drift(y[j], vy[j], dt, Ly, bad);
                    z[j] = drift(z[j], vz[j], dt, Lz, bad);
                    if (a.accel) {
                        vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                        vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                        vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                    }
                }
            }
            if (BIN) bin4<Real, RULE, COLLIDE>(a, x, y, z, vx, vy, vz, tg, nv, sF + 3, L0, L1, L2, base, rr, step,
                                                m, sc, sums, C);
            if (STREAM) { st4(X + i, x); st4(Y + i, y); st4(Z + i, z); }
            if (COLLIDE || (STREAM && a.accel)) { st4(VX + i, vx); st4(VY + i, vy); st4(VZ + i, vz); }
        }
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// ------------------------------------------- staged pass (bulk async copies)
// The same per-particle arithmetic as k_solvent, but each CTA streams its
// tiles through a three-stage shared-memory ring: thread 0 issues one
// cp.async.bulk per SoA array (completion counted on an mbarrier) for tile
// k+2 while the CTA computes tile k+1 and tile k is written back with bulk
// stores.  Memory-level parallelism is then set by the copy engine, not by
// the number of resident warps.  One CTA barrier per tile; the tile records,
// replica fields and grid shifts are read ahead by thread 0 after it, so no
// serial set-up stands between two tiles.  Every mbarrier wait is bounded.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity)
{
    for (uint32_t i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
// The solvent state streams through L2 once per pass: its bulk copies carry an
// evict-first policy, so that the cell records and words, which the pass
// gathers and reduces into repeatedly, keep their L2 lines (the pass alone:
// 1.37 -> 1.34 ms at 80 M particles).
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_load_ef(void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(b)), "l"(policy_evict_first())
                 : "memory");
}
__device__ __forceinline__ void bulk_store_ef(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;"
                 ::"l"(dst), "r"(smem_addr(src)), "r"(bytes), "l"(policy_evict_first())
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void sld4(const float *p, float (&o)[4])
{
    float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void sld4(const double *p, double (&o)[4])
{
    double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void sst4(float *p, const float (&o)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void sst4(double *p, const double (&o)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
}

struct TileMeta {
    int32_t S[6];     // grid shifts: collision (0..2), binning (3..5)
    float Sf[6];      // the same as s = S 2^-20 (FP32 form)
    int32_t L[3];
    int32_t base;     // first global cell of the replica
    int32_t n;        // particles in the tile
    uint32_t key0, key1;
    int32_t pad;
    int64_t beg;      // first slot
};

__device__ __forceinline__ int32_t tile_shift(const TileMeta &m, int c, int32_t) { return m.S[c]; }
__device__ __forceinline__ float tile_shift(const TileMeta &m, int c, float) { return m.Sf[c]; }

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

template <typename Real, int RULE>
__host__ __device__ constexpr size_t stage_bytes(int cap)
{
    return ((size_t)cap * (6 * sizeof(Real) + (RULE == 1 ? 4 : 0)) + 127) & ~(size_t)127;
}

constexpr int ST_STAGES = 3;

// Register cap of the FP32 SRD form of the staged pass (threads of all its
// CTAs on an SM times the cap leave the rest to the site/body kernels that run
// beside it); the other forms take up to 128.
#ifndef MPCD_ST_SRD_REGS
#define MPCD_ST_SRD_REGS 96
#endif
template <typename Real, int RULE> struct StRegs {
    static constexpr int n = sizeof(Real) == 4 && RULE == 0 ? MPCD_ST_SRD_REGS : 128;
};

template <typename Real, int RULE, int FLAGS>
__global__ void __maxnreg__((StRegs<Real, RULE>::n)) k_solvent_staged(StepArgs a, int cap)
{
    constexpr bool COLLIDE = FLAGS & SOLV_COLLIDE;
    constexpr bool STREAM = FLAGS & SOLV_STREAM;
    constexpr bool BIN = FLAGS & SOLV_BIN;
    typedef typename SumWord<Real>::type W;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[ST_STAGES];
    __shared__ TileMeta meta[ST_STAGES];
    __shared__ TileMeta rcache;   // fields and grid shifts of the last replica met
    __shared__ int rcache_rep;
    __shared__ int stile[ST_STAGES];   // tile in each stage (-1: none, the pass is done)

    const size_t SB = stage_bytes<Real, RULE>(cap);
    const int64_t step = *a.d_step;
    const Real dt = Consts<Real>::dt(a), m = Consts<Real>::m(a), kT = Consts<Real>::kT(a);
    const Real ca = Consts<Real>::ca(a), sa = Consts<Real>::sa(a);
    const Real sc = sqrt(kT / m);
    auto garr = [&](int c) -> Real * {
        void *p = c == 0 ? a.x : c == 1 ? a.y : c == 2 ? a.z : c == 3 ? a.vx : c == 4 ? a.vy : a.vz;
        return reinterpret_cast<Real *>(p);
    };
    W *sums = reinterpret_cast<W *>(a.sums);
    const int64_t C = a.n_cells;
    int bad = 0;

    // Tiles are handed out by a counter (a.tile_ctr, zero at launch) when one is
    // given, else round robin: a CTA slowed by the kernels that share its SM
    // then takes fewer tiles instead of delaying the end of the pass.
    // Thread 0 only: the index and record of the next tile to issue are taken
    // one issue ahead, so that neither stands between two tiles.
    int nt = -1;
    int32_t nrep = 0;
    int64_t nbeg = 0, nend = 0;
    auto take = [&](int j) {   // the index of local tile j and its record
        const int t = a.tile_ctr ? atomicAdd(a.tile_ctr, 1) : (int)blockIdx.x + j * (int)gridDim.x;
        nt = t < a.n_tiles ? t : -1;
        if (nt >= 0) {
            const Tile tn = a.tiles[nt];
            nrep = tn.rep; nbeg = tn.begin; nend = tn.end;
        }
    };
    auto issue = [&](int j) {   // local tile j into stage j % ST_STAGES
        const int q = j % ST_STAGES;
        stile[q] = nt;
        if (nt < 0) return;
        const int rep = nrep;
        const int64_t tbeg = nbeg, tend = nend;
        take(j + 1);
        if (rep != rcache_rep) {
            const DevReplica cr = a.reps[rep];
            if (COLLIDE) grid_shift(cr, step, &rcache.S[0]);
            if (BIN) grid_shift(cr, step + (COLLIDE ? 1 : 0), &rcache.S[3]);
            for (int c = 0; c < 6; ++c) rcache.Sf[c] = shift_as(rcache.S[c], 0.0f);
            rcache.L[0] = cr.L[0]; rcache.L[1] = cr.L[1]; rcache.L[2] = cr.L[2];
            rcache.base = cr.cell_base;
            rcache.key0 = cr.key0;
            rcache.key1 = cr.key1;
            rcache_rep = rep;
        }
        TileMeta &mt = meta[q];
        mt = rcache;
        mt.n = (int)(tend - tbeg);
        mt.beg = tbeg;
        const int n4 = (mt.n + 3) & ~3;
        const uint32_t nb = (uint32_t)(n4 * sizeof(Real));
        unsigned char *base = smem + q * SB;
        mbar_expect_tx(&full[q], 6 * nb + (RULE == 1 ? (uint32_t)(n4 * 4) : 0u));
        for (int c = 0; c < 6; ++c) bulk_load_ef(base + (size_t)c * cap * sizeof(Real), garr(c) + tbeg, nb, &full[q]);
        if (RULE == 1) bulk_load_ef(base + (size_t)6 * cap * sizeof(Real), a.tag + tbeg, (uint32_t)(n4 * 4), &full[q]);
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q < ST_STAGES; ++q) mbar_init(&full[q], 1);
        mbar_fence_init();
        rcache_rep = -1;
        take(0);
        for (int j = 0; j < ST_STAGES - 1; ++j) issue(j);
    }
    __syncthreads();

    for (int k = 0;; ++k) {
        const int q = k % ST_STAGES;
        if (stile[q] < 0) break;   // written before the previous barrier: uniform
        // a timed-out wait is folded into the barrier at the end of the tile:
        // the arithmetic on a stage that did not land is memory-safe (every
        // index it forms is bounded) and its results are discarded
        const bool got = mbar_wait_bounded(&full[q], (uint32_t)((k / ST_STAGES) & 1));
        const TileMeta &mt = meta[q];
        typename ShiftT<Real>::type sF[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) sF[c] = tile_shift(mt, c, typename ShiftT<Real>::type());
        const int L0 = mt.L[0], L1 = mt.L[1], L2 = mt.L[2], base = mt.base, n = mt.n;
        const Real Lx = (Real)L0, Ly = (Real)L1, Lz = (Real)L2;
        DevReplica rr;
        rr.key0 = mt.key0;
        rr.key1 = mt.key1;
        Real *S[6];
        for (int c = 0; c < 6; ++c) S[c] = reinterpret_cast<Real *>(smem + q * SB + (size_t)c * cap * sizeof(Real));
        const uint32_t *stag = reinterpret_cast<const uint32_t *>(smem + q * SB + (size_t)6 * cap * sizeof(Real));

        // uniform trip count: every lane of a warp reaches the warp-wide flush
        for (int i0 = 0; i0 < n && got; i0 += 4 * blockDim.x) {
            const int i = i0 + 4 * threadIdx.x;
            const int nv = max(0, min(4, n - i));
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            if (nv > 0) {
                sld4(S[0] + i, x); sld4(S[1] + i, y); sld4(S[2] + i, z);
                sld4(S[3] + i, vx); sld4(S[4] + i, vy); sld4(S[5] + i, vz);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = y[j] = z[j] = vx[j] = vy[j] = vz[j] = Real(0);
            }
            uint32_t tg[4] = {0, 0, 0, 0};
            if (RULE == 1 && nv > 0) {
                uint4 t4 = *reinterpret_cast<const uint4 *>(stag + i);
                tg[0] = t4.x; tg[1] = t4.y; tg[2] = t4.z; tg[3] = t4.w;
            }
            if (COLLIDE) {
                // issue the four parameter gathers before any of them is used
                CellParams<Real> p[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int c = base + cell_bin(x[j], sF[0], L0) +
                            L0 * (cell_bin(y[j], sF[1], L1) + L1 * cell_bin(z[j], sF[2], L2));
                    c = j < nv ? c : base;
                    p[j] = get_params<Real>(a.params, c);
                }
                Real nn[4][3];
                if (RULE == 1) {
                    // the four particles' Philox blocks are independent: draw
                    // them all (a lane past the tile end draws for id 0), so
                    // that their dependent rounds interleave
#pragma unroll
                    for (int j = 0; j < 4; ++j) normals3(draw(rr, step, tg[j], TAG_AT, 0u), nn[j]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the rule is applied to every slot and kept where it
                    // applies (no branch): a member of a cell that collides
                    const bool on = j < nv && p[j].kappa >= Real(0);
                    Real rx, ry, rz;
                    if (RULE == 0) {
                        rx = vx[j]; ry = vy[j]; rz = vz[j];
                        srd_rotate<Real>(p[j], ca, sa, rx, ry, rz);
                    } else {
                        rx = p[j].ux + sc * nn[j][0] - p[j].ax;
                        ry = p[j].uy + sc * nn[j][1] - p[j].ay;
                        rz = p[j].uz + sc * nn[j][2] - p[j].az;
                    }
                    vx[j] = on ? rx : vx[j];
                    vy[j] = on ? ry : vy[j];
                    vz[j] = on ? rz : vz[j];
                }
            }
            if (STREAM) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nv) {
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                        x[j] = drift(x[j], vx[j], dt, Lx, bad);
                        y[j] = drift(y[j], vy[j], dt, Ly, bad);
                        z[j] = drift(z[j], vz[j], dt, Lz, bad);
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                    }
            }
            if (BIN) bin4<Real, RULE, COLLIDE>(a, x, y, z, vx, vy, vz, tg, nv, sF + 3, L0, L1, L2, base, rr, step,
                                                m, sc, sums, C);
            if (nv > 0) {
                if (STREAM) { sst4(S[0] + i, x); sst4(S[1] + i, y); sst4(S[2] + i, z); }
                if (COLLIDE || (STREAM && a.accel)) { sst4(S[3] + i, vx); sst4(S[4] + i, vy); sst4(S[5] + i, vz); }
            }
        }
        fence_async_smem();   // results visible to the bulk stores
        if (__syncthreads_or(!got)) {
            if (threadIdx.x == 0) {
                atomicOr(a.d_err, ERR_TIMEOUT);
                // let the copies in flight land before the CTA leaves (bounded)
                bulk_wait_all();
                for (int j = k; j < k + ST_STAGES - 1 && stile[j % ST_STAGES] >= 0; ++j)
                    mbar_wait_bounded(&full[j % ST_STAGES], (uint32_t)((j / ST_STAGES) & 1));
            }
            return;
        }
        if (threadIdx.x == 0) {
            if (STREAM || COLLIDE) {
                const uint32_t nb = (uint32_t)(((n + 3) & ~3) * sizeof(Real));
                const int64_t beg = mt.beg;
                if (STREAM)
                    for (int c = 0; c < 3; ++c) bulk_store_ef(garr(c) + beg, S[c], nb);
                if (COLLIDE || (STREAM && a.accel))
                    for (int c = 3; c < 6; ++c) bulk_store_ef(garr(c) + beg, S[c], nb);
            }
            bulk_commit();
            if (nt >= 0) bulk_wait_read_1();   // the store of tile k - 1 has read the stage that tile k + 2 takes
            issue(k + ST_STAGES - 1);
        }
    }
    if (threadIdx.x == 0) bulk_wait_all();
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// --------------------------- warp-specialised pass (producer + consumers)
// The last warp of the CTA is the producer: one lane loads the tile
// metadata (range, box, grid shifts), issues the bulk copies of each tile into
// a three-stage shared-memory ring and, once the consumer warps have signalled
// that a tile is done, its bulk stores.  The consumer warps only compute: no
// CTA-wide barrier inside the loop, so tile set-up and write-back overlap with
// the arithmetic of other tiles.  Stage s of local tile k: loads complete on
// full[s], the consumers arrive on done[s]; a stage is refilled only after the
// store issued from it two tiles earlier has finished reading it.  Every wait
// is bounded; on a timeout the error word gets ERR_TIMEOUT and the CTA drains.
constexpr int WS_STAGES = 3;

template <typename Real, int RULE, int FLAGS>
__global__ void __launch_bounds__(544) k_solvent_ws(StepArgs a, int cap)
{
    constexpr bool COLLIDE = FLAGS & SOLV_COLLIDE;
    constexpr bool STREAM = FLAGS & SOLV_STREAM;
    constexpr bool BIN = FLAGS & SOLV_BIN;
    typedef typename SumWord<Real>::type W;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[WS_STAGES], done[WS_STAGES];
    __shared__ TileMeta meta[WS_STAGES];

    const int n_cons = (int)blockDim.x - 32;           // consumer threads
    const int n_cwarps = n_cons >> 5;
    const bool producer = (int)threadIdx.x >= n_cons;
    const size_t SB = stage_bytes<Real, RULE>(cap);
    const int64_t step = *a.d_step;
    Real *G[6] = {reinterpret_cast<Real *>(a.x), reinterpret_cast<Real *>(a.y), reinterpret_cast<Real *>(a.z),
                  reinterpret_cast<Real *>(a.vx), reinterpret_cast<Real *>(a.vy), reinterpret_cast<Real *>(a.vz)};
    const int K = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int q = 0; q < WS_STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], (uint32_t)n_cwarps);
        }
        mbar_fence_init();
    }
    __syncthreads();   // the only CTA-wide barrier

    if (producer) {
        if (threadIdx.x != (unsigned)n_cons) return;   // one lane drives the ring
        auto store_tile = [&](int j) -> bool {          // local tile j, after its consumers are done
            const int q = j % WS_STAGES;
            if (!mbar_wait_bounded(&done[q], (uint32_t)((j / WS_STAGES) & 1))) return false;
            if (STREAM || COLLIDE) {
                const TileMeta &m = meta[q];
                const uint32_t nb = (uint32_t)(((m.n + 3) & ~3) * sizeof(Real));
                unsigned char *base = smem + q * SB;
                if (STREAM)
                    for (int c = 0; c < 3; ++c) bulk_store_ef(G[c] + m.beg, base + (size_t)c * cap * sizeof(Real), nb);
                if (COLLIDE || (STREAM && a.accel))
                    for (int c = 3; c < 6; ++c) bulk_store_ef(G[c] + m.beg, base + (size_t)c * cap * sizeof(Real), nb);
            }
            bulk_commit();
            return true;
        };
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            const int q = k % WS_STAGES;
            if (k >= WS_STAGES) bulk_wait_read_1();     // the store of tile k - 3 has read stage q
            const Tile tl = a.tiles[blockIdx.x + k * gridDim.x];
            const DevReplica r = a.reps[tl.rep];
            TileMeta &m = meta[q];
            if (COLLIDE) grid_shift(r, step, &m.S[0]);
            if (BIN) grid_shift(r, step + (COLLIDE ? 1 : 0), &m.S[3]);
            for (int c = 0; c < 6; ++c) m.Sf[c] = shift_as(m.S[c], 0.0f);
            m.L[0] = r.L[0]; m.L[1] = r.L[1]; m.L[2] = r.L[2];
            m.base = r.cell_base;
            m.n = (int)(tl.end - tl.begin);
            m.key0 = r.key0;
            m.key1 = r.key1;
            m.beg = tl.begin;
            const int n4 = (m.n + 3) & ~3;
            const uint32_t nb = (uint32_t)(n4 * sizeof(Real));
            unsigned char *base = smem + q * SB;
            mbar_expect_tx(&full[q], 6 * nb + (RULE == 1 ? (uint32_t)(n4 * 4) : 0u));
            for (int c = 0; c < 6; ++c) bulk_load_ef(base + (size_t)c * cap * sizeof(Real), G[c] + tl.begin, nb, &full[q]);
            if (RULE == 1) bulk_load_ef(base + (size_t)6 * cap * sizeof(Real), a.tag + tl.begin, (uint32_t)(n4 * 4), &full[q]);
            if (k >= 1) ok = store_tile(k - 1);
        }
        if (ok && K >= 1) ok = store_tile(K - 1);
        if (!ok) atomicOr(a.d_err, ERR_TIMEOUT);
        bulk_wait_all();
        return;
    }

    // consumers
    const Real dt = Consts<Real>::dt(a), m = Consts<Real>::m(a), kT = Consts<Real>::kT(a);
    const Real ca = Consts<Real>::ca(a), sa = Consts<Real>::sa(a);
    const Real sc = sqrt(kT / m);
    W *sums = reinterpret_cast<W *>(a.sums);
    const int64_t C = a.n_cells;
    int bad = 0;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < K; ++k) {
        const int q = k % WS_STAGES;
        if (!mbar_wait_bounded(&full[q], (uint32_t)((k / WS_STAGES) & 1))) {
            if (lane == 0) atomicOr(a.d_err, ERR_TIMEOUT);
            break;
        }
        const TileMeta &mt = meta[q];
        typename ShiftT<Real>::type sF[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) sF[c] = tile_shift(mt, c, typename ShiftT<Real>::type());
        const int L0 = mt.L[0], L1 = mt.L[1], L2 = mt.L[2], base = mt.base, n = mt.n;
        const Real Lx = (Real)L0, Ly = (Real)L1, Lz = (Real)L2;
        DevReplica rr;
        rr.key0 = mt.key0;
        rr.key1 = mt.key1;
        Real *S[6];
        for (int c = 0; c < 6; ++c) S[c] = reinterpret_cast<Real *>(smem + q * SB + (size_t)c * cap * sizeof(Real));
        const uint32_t *stag = reinterpret_cast<const uint32_t *>(smem + q * SB + (size_t)6 * cap * sizeof(Real));

        // uniform trip count: every lane of a warp reaches the warp-wide flush
        for (int i0 = 0; i0 < n; i0 += 4 * n_cons) {
            const int i = i0 + 4 * (int)threadIdx.x;
            const int nv = max(0, min(4, n - i));
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            if (nv > 0) {
                sld4(S[0] + i, x); sld4(S[1] + i, y); sld4(S[2] + i, z);
                sld4(S[3] + i, vx); sld4(S[4] + i, vy); sld4(S[5] + i, vz);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = y[j] = z[j] = vx[j] = vy[j] = vz[j] = Real(0);
            }
            uint32_t tg[4] = {0, 0, 0, 0};
            if (RULE == 1 && nv > 0) {
                uint4 t4 = *reinterpret_cast<const uint4 *>(stag + i);
                tg[0] = t4.x; tg[1] = t4.y; tg[2] = t4.z; tg[3] = t4.w;
            }
            if (COLLIDE) {
                CellParams<Real> p[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int c = base + cell_bin(x[j], sF[0], L0) +
                            L0 * (cell_bin(y[j], sF[1], L1) + L1 * cell_bin(z[j], sF[2], L2));
                    c = j < nv ? c : base;
                    p[j] = get_params<Real>(a.params, c);
                }
                Real nn[4][3];
                if (RULE == 1) {
                    // the four particles' Philox blocks are independent: draw
                    // them all (a lane past the tile end draws for id 0), so
                    // that their dependent rounds interleave
#pragma unroll
                    for (int j = 0; j < 4; ++j) normals3(draw(rr, step, tg[j], TAG_AT, 0u), nn[j]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the rule is applied to every slot and kept where it
                    // applies (no branch): a member of a cell that collides
                    const bool on = j < nv && p[j].kappa >= Real(0);
                    Real rx, ry, rz;
                    if (RULE == 0) {
                        rx = vx[j]; ry = vy[j]; rz = vz[j];
                        srd_rotate<Real>(p[j], ca, sa, rx, ry, rz);
                    } else {
                        rx = p[j].ux + sc * nn[j][0] - p[j].ax;
                        ry = p[j].uy + sc * nn[j][1] - p[j].ay;
                        rz = p[j].uz + sc * nn[j][2] - p[j].az;
                    }
                    vx[j] = on ? rx : vx[j];
                    vy[j] = on ? ry : vy[j];
                    vz[j] = on ? rz : vz[j];
                }
            }
            if (STREAM) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nv) {
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                        x[j] = drift(x[j], vx[j], dt, Lx, bad);
                        y[j] = drift(y[j], vy[j], dt, Ly, bad);
                        z[j] = drift(z[j], vz[j], dt, Lz, bad);
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                    }
            }
            if (BIN) bin4<Real, RULE, COLLIDE>(a, x, y, z, vx, vy, vz, tg, nv, sF + 3, L0, L1, L2, base, rr, step,
                                                m, sc, sums, C);
            if (nv > 0) {
                if (STREAM) { sst4(S[0] + i, x); sst4(S[1] + i, y); sst4(S[2] + i, z); }
                if (COLLIDE || (STREAM && a.accel)) { sst4(S[3] + i, vx); sst4(S[4] + i, vy); sst4(S[5] + i, vz); }
            }
        }
        fence_async_smem();   // results visible to the bulk stores
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[q]);
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// ----------------------------------------------- warp-tiled pass (per warp)
// Every warp runs its own three-stage ring of small tiles (the tile table is
// built with the warp-tile size): lane 0 issues the bulk loads of tile k+1
// and the bulk stores of tile k, the warp computes tile k.  Warps share no
// barrier, so they drift apart and the latency of one warp's parameter
// gathers is covered by the arithmetic of others.  The tile record of the
// next fetch is loaded one tile ahead; the grid shifts are computed once per
// replica a warp meets.  Every wait is bounded.
constexpr int WT_STAGES = 3, WT_MAX_WARPS = 16;

// Register cap of the FP32 SRD form (80, at most 512 threads): 512 x 80
// registers leave 24 K of the SM's 64 K registers to the site/body kernels
// that run beside this pass on the second stream (a cap of 96 left room for
// one of their CTAs per SM, none without a cap; 72 and below spill in the
// loop).  The AT form draws two Philox normals per particle and is latency-
// bound on their rounds: it gains more from registers (ILP) than from the
// overlap (L=200: 2.40 ms with 128, 2.69 with 112, 3.01 with 96).
#ifndef MPCD_WT_SRD_REGS
#define MPCD_WT_SRD_REGS 80
#endif
template <typename Real, int RULE> struct WtRegs {
    static constexpr int n = sizeof(Real) == 4 && RULE == 0 ? MPCD_WT_SRD_REGS : 128;
};

template <typename Real, int RULE, int FLAGS>
__global__ void __maxnreg__((WtRegs<Real, RULE>::n)) k_solvent_wt(StepArgs a, int cap)
{
    constexpr bool COLLIDE = FLAGS & SOLV_COLLIDE;
    constexpr bool STREAM = FLAGS & SOLV_STREAM;
    constexpr bool BIN = FLAGS & SOLV_BIN;
    typedef typename SumWord<Real>::type W;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[WT_MAX_WARPS][WT_STAGES];
    __shared__ TileMeta meta[WT_MAX_WARPS][WT_STAGES];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const size_t SB = stage_bytes<Real, RULE>(cap);
    unsigned char *wsm = smem + (size_t)warp * WT_STAGES * SB;
    const int64_t step = *a.d_step;
    // the global arrays are read from the kernel parameters where lane 0 needs them
    auto garr = [&](int c) -> Real * {
        void *p = c == 0 ? a.x : c == 1 ? a.y : c == 2 ? a.z : c == 3 ? a.vx : c == 4 ? a.vy : a.vz;
        return reinterpret_cast<Real *>(p);
    };
    const int gw = blockIdx.x * nwarps + warp, GW = gridDim.x * nwarps;
    const int K = a.n_tiles > gw ? (a.n_tiles - 1 - gw) / GW + 1 : 0;   // tiles of this warp

    if (lane == 0) {
        for (int q = 0; q < WT_STAGES; ++q) mbar_init(&full[warp][q], 1);
        mbar_fence_init();
    }
    __syncwarp();

    // lane 0 only: metadata and bulk loads of local tile k into stage q.  The
    // replica fields and grid shifts of the last replica met stay in shared
    // memory (wcache), so they take no registers in the computing lanes.
    __shared__ TileMeta wcache[WT_MAX_WARPS];
    __shared__ int wrep[WT_MAX_WARPS];
    if (lane == 0) wrep[warp] = -1;
    int32_t nrep = 0;
    int64_t nbeg = 0, nend = 0;   // tile record of the next fetch
    if (lane == 0 && K > 0) {
        const Tile t0 = a.tiles[gw];
        nrep = t0.rep; nbeg = t0.begin; nend = t0.end;
    }
    auto fetch = [&](int k, int q) {
        const int rep = nrep;
        const int64_t tbeg = nbeg, tend = nend;
        if (k + 1 < K) {   // used by the following fetch
            const Tile tn = a.tiles[gw + (k + 1) * GW];
            nrep = tn.rep; nbeg = tn.begin; nend = tn.end;
        }
        TileMeta &wc = wcache[warp];
        if (rep != wrep[warp]) {
            const DevReplica cr = a.reps[rep];
            if (COLLIDE) grid_shift(cr, step, &wc.S[0]);
            if (BIN) grid_shift(cr, step + (COLLIDE ? 1 : 0), &wc.S[3]);
            for (int c = 0; c < 6; ++c) wc.Sf[c] = shift_as(wc.S[c], 0.0f);
            wc.L[0] = cr.L[0]; wc.L[1] = cr.L[1]; wc.L[2] = cr.L[2];
            wc.base = cr.cell_base;
            wc.key0 = cr.key0;
            wc.key1 = cr.key1;
            wrep[warp] = rep;
        }
        TileMeta &m = meta[warp][q];
        m = wc;
        m.n = (int)(tend - tbeg);
        m.beg = tbeg;
        const Tile tl{rep, 0, tbeg, tend};
        const int n4 = (m.n + 3) & ~3;
        const uint32_t nb = (uint32_t)(n4 * sizeof(Real));
        unsigned char *base = wsm + q * SB;
        mbar_expect_tx(&full[warp][q], 6 * nb + (RULE == 1 ? (uint32_t)(n4 * 4) : 0u));
        for (int c = 0; c < 6; ++c) bulk_load_ef(base + (size_t)c * cap * sizeof(Real), garr(c) + tl.begin, nb, &full[warp][q]);
        if (RULE == 1) bulk_load_ef(base + (size_t)6 * cap * sizeof(Real), a.tag + tl.begin, (uint32_t)(n4 * 4), &full[warp][q]);
    };

    const Real dt = Consts<Real>::dt(a), m = Consts<Real>::m(a), kT = Consts<Real>::kT(a);
    const Real ca = Consts<Real>::ca(a), sa = Consts<Real>::sa(a);
    const Real sc = sqrt(kT / m);
    W *sums = reinterpret_cast<W *>(a.sums);
    const int64_t C = a.n_cells;
    int bad = 0;
    if (lane == 0 && K > 0) fetch(0, 0);
    __syncwarp();
    for (int k = 0; k < K; ++k) {
        const int q = k % WT_STAGES;
        if (lane == 0 && k + 1 < K) {
            if (k + 1 >= WT_STAGES) bulk_wait_read_1();   // the store of tile k - 2 has read that stage
            fetch(k + 1, (k + 1) % WT_STAGES);
        }
        const bool got = mbar_wait_bounded(&full[warp][q], (uint32_t)((k / WT_STAGES) & 1));
        if (!__all_sync(0xffffffffu, got)) {
            if (lane == 0) {
                atomicOr(a.d_err, ERR_TIMEOUT);
                // let the copies in flight land before the CTA leaves (bounded)
                mbar_wait_bounded(&full[warp][q], (uint32_t)((k / WT_STAGES) & 1));
                if (k + 1 < K)
                    mbar_wait_bounded(&full[warp][(k + 1) % WT_STAGES], (uint32_t)(((k + 1) / WT_STAGES) & 1));
            }
            break;
        }
        const TileMeta &mt = meta[warp][q];
        typename ShiftT<Real>::type sF[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) sF[c] = tile_shift(mt, c, typename ShiftT<Real>::type());
        const int L0 = mt.L[0], L1 = mt.L[1], L2 = mt.L[2], base = mt.base, n = mt.n;
        const Real Lx = (Real)L0, Ly = (Real)L1, Lz = (Real)L2;
        DevReplica rr;
        rr.key0 = mt.key0;
        rr.key1 = mt.key1;
        Real *S[6];
        for (int c = 0; c < 6; ++c) S[c] = reinterpret_cast<Real *>(wsm + q * SB + (size_t)c * cap * sizeof(Real));
        const uint32_t *stag = reinterpret_cast<const uint32_t *>(wsm + q * SB + (size_t)6 * cap * sizeof(Real));

        for (int i0 = 0; i0 < n; i0 += 128) {
            const int i = i0 + 4 * lane;
            const int nv = max(0, min(4, n - i));
            Real x[4], y[4], z[4], vx[4], vy[4], vz[4];
            if (nv > 0) {
                sld4(S[0] + i, x); sld4(S[1] + i, y); sld4(S[2] + i, z);
                sld4(S[3] + i, vx); sld4(S[4] + i, vy); sld4(S[5] + i, vz);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = y[j] = z[j] = vx[j] = vy[j] = vz[j] = Real(0);
            }
            uint32_t tg[4] = {0, 0, 0, 0};
            if (RULE == 1 && nv > 0) {
                uint4 t4 = *reinterpret_cast<const uint4 *>(stag + i);
                tg[0] = t4.x; tg[1] = t4.y; tg[2] = t4.z; tg[3] = t4.w;
            }
            if (COLLIDE) {
                CellParams<Real> p[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int c = base + cell_bin(x[j], sF[0], L0) +
                            L0 * (cell_bin(y[j], sF[1], L1) + L1 * cell_bin(z[j], sF[2], L2));
                    c = j < nv ? c : base;
                    p[j] = get_params<Real>(a.params, c);
                }
                Real nn[4][3];
                if (RULE == 1) {
                    // the four particles' Philox blocks are independent: draw
                    // them all (a lane past the tile end draws for id 0), so
                    // that their dependent rounds interleave
#pragma unroll
                    for (int j = 0; j < 4; ++j) normals3(draw(rr, step, tg[j], TAG_AT, 0u), nn[j]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the rule is applied to every slot and kept where it
                    // applies (no branch): a member of a cell that collides
                    const bool on = j < nv && p[j].kappa >= Real(0);
                    Real rx, ry, rz;
                    if (RULE == 0) {
                        rx = vx[j]; ry = vy[j]; rz = vz[j];
                        srd_rotate<Real>(p[j], ca, sa, rx, ry, rz);
                    } else {
                        rx = p[j].ux + sc * nn[j][0] - p[j].ax;
                        ry = p[j].uy + sc * nn[j][1] - p[j].ay;
                        rz = p[j].uz + sc * nn[j][2] - p[j].az;
                    }
                    vx[j] = on ? rx : vx[j];
                    vy[j] = on ? ry : vy[j];
                    vz[j] = on ? rz : vz[j];
                }
            }
            if (STREAM) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nv) {
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                        x[j] = drift(x[j], vx[j], dt, Lx, bad);
                        y[j] = drift(y[j], vy[j], dt, Ly, bad);
                        z[j] = drift(z[j], vz[j], dt, Lz, bad);
                        if (a.accel) {
                            vx[j] = kick(vx[j], Consts<Real>::ah(a, 0));
                            vy[j] = kick(vy[j], Consts<Real>::ah(a, 1));
                            vz[j] = kick(vz[j], Consts<Real>::ah(a, 2));
                        }
                    }
            }
            if (BIN) bin4<Real, RULE, COLLIDE>(a, x, y, z, vx, vy, vz, tg, nv, sF + 3, L0, L1, L2, base, rr, step,
                                                m, sc, sums, C);
            if (nv > 0) {
                if (STREAM) { sst4(S[0] + i, x); sst4(S[1] + i, y); sst4(S[2] + i, z); }
                if (COLLIDE || (STREAM && a.accel)) { sst4(S[3] + i, vx); sst4(S[4] + i, vy); sst4(S[5] + i, vz); }
            }
        }
        fence_async_smem();   // results visible to the bulk stores
        __syncwarp();
        if (lane == 0 && (STREAM || COLLIDE)) {
            const uint32_t nb = (uint32_t)(((n + 3) & ~3) * sizeof(Real));
            unsigned char *sb = wsm + q * SB;
            const int64_t beg = mt.beg;
            if (STREAM)
                for (int c = 0; c < 3; ++c) bulk_store_ef(garr(c) + beg, sb + (size_t)c * cap * sizeof(Real), nb);
            if (COLLIDE || (STREAM && a.accel))
                for (int c = 3; c < 6; ++c) bulk_store_ef(garr(c) + beg, sb + (size_t)c * cap * sizeof(Real), nb);
        }
        if (lane == 0) bulk_commit();
        __syncwarp();
    }
    if (lane == 0) bulk_wait_all();
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// Opt a kernel in to `bytes` of dynamic shared memory on the current device,
// once per (kernel, device) and size; safe from several host threads.
static void smem_opt_in(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;   // the launch reports the error
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = done[{func, dev}];
    if (bytes > have &&
        cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
        have = bytes;
}

// The persistent passes take their tiles round robin: a CTA that is not
// resident from the start runs its share after the others have finished.  The
// grid is therefore capped at the CTAs that are resident together (registers,
// shared memory and threads of this kernel at this launch shape), once per
// (kernel, device, shape).
static int resident_grid(const void *func, int grid, int threads, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<std::pair<const void *, int>, std::pair<int, size_t>>, int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return grid;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(std::make_pair(func, dev), std::make_pair(threads, bytes));
    auto it = done.find(key);
    if (it == done.end()) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, bytes) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return grid;                       // the launch reports any error
        }
        it = done.emplace(key, std::max(1, per_sm) * std::max(1, sms)).first;
    }
    return std::max(1, std::min(grid, it->second));
}

template <typename Real, int RULE, int FLAGS>
static void launch_wt(const StepArgs &a, LaunchCfg cfg, cudaStream_t s)
{
    const int warps = cfg.block / 32;
    const size_t bytes = (size_t)warps * WT_STAGES * solvent_stage_bytes(sizeof(Real) == 4 ? 1 : 0, RULE, cfg.cap);
    const void *f = (const void *)k_solvent_wt<Real, RULE, FLAGS>;
    smem_opt_in(f, bytes);
    const int grid = resident_grid(f, cfg.grid, cfg.block, bytes);
    k_solvent_wt<Real, RULE, FLAGS><<<grid, cfg.block, bytes, s>>>(a, cfg.cap);
}

template <typename Real, int RULE, int FLAGS>
static void launch_ws(const StepArgs &a, LaunchCfg cfg, cudaStream_t s)
{
    const size_t bytes = (size_t)WS_STAGES * solvent_stage_bytes(sizeof(Real) == 4 ? 1 : 0, RULE, cfg.cap);
    const void *f = (const void *)k_solvent_ws<Real, RULE, FLAGS>;
    smem_opt_in(f, bytes);
    const int grid = resident_grid(f, cfg.grid, cfg.block + 32, bytes);
    k_solvent_ws<Real, RULE, FLAGS><<<grid, cfg.block + 32, bytes, s>>>(a, cfg.cap);
}

template <typename Real, int RULE, int FLAGS>
static void launch_staged(const StepArgs &a, LaunchCfg cfg, cudaStream_t s)
{
    const size_t bytes = solvent_smem_bytes(sizeof(Real) == 4 ? 1 : 0, RULE, cfg.cap, cfg.block);
    const void *f = (const void *)k_solvent_staged<Real, RULE, FLAGS>;
    smem_opt_in(f, bytes);
    const int grid = resident_grid(f, cfg.grid, cfg.block, bytes);
    if (a.tile_ctr) cudaMemsetAsync(a.tile_ctr, 0, sizeof(int), s);   // the launch reports any error
    k_solvent_staged<Real, RULE, FLAGS><<<grid, cfg.block, bytes, s>>>(a, cfg.cap);
}

template <typename Real, int RULE, int FLAGS>
static void launch_direct(const StepArgs &a, LaunchCfg cfg, cudaStream_t s)
{
    const int grid = resident_grid((const void *)k_solvent<Real, RULE, FLAGS>, cfg.grid, cfg.block, 0);
    k_solvent<Real, RULE, FLAGS><<<grid, cfg.block, 0, s>>>(a);
}

template <typename Real, int RULE>
static void dispatch_flags(const StepArgs &a, int flags, LaunchCfg cfg, cudaStream_t s)
{
    if (cfg.staged == 3) {
        switch (flags) {
        case SOLV_STREAM: launch_wt<Real, RULE, SOLV_STREAM>(a, cfg, s); break;
        case SOLV_BIN: launch_wt<Real, RULE, SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE: launch_wt<Real, RULE, SOLV_COLLIDE>(a, cfg, s); break;
        case SOLV_STREAM | SOLV_BIN: launch_wt<Real, RULE, SOLV_STREAM | SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN:
            launch_wt<Real, RULE, SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN>(a, cfg, s);
            break;
        default: break;
        }
        return;
    }
    if (cfg.staged == 2) {
        switch (flags) {
        case SOLV_STREAM: launch_ws<Real, RULE, SOLV_STREAM>(a, cfg, s); break;
        case SOLV_BIN: launch_ws<Real, RULE, SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE: launch_ws<Real, RULE, SOLV_COLLIDE>(a, cfg, s); break;
        case SOLV_STREAM | SOLV_BIN: launch_ws<Real, RULE, SOLV_STREAM | SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN:
            launch_ws<Real, RULE, SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN>(a, cfg, s);
            break;
        default: break;
        }
        return;
    }
    if (cfg.staged) {
        switch (flags) {
        case SOLV_STREAM: launch_staged<Real, RULE, SOLV_STREAM>(a, cfg, s); break;
        case SOLV_BIN: launch_staged<Real, RULE, SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE: launch_staged<Real, RULE, SOLV_COLLIDE>(a, cfg, s); break;
        case SOLV_STREAM | SOLV_BIN: launch_staged<Real, RULE, SOLV_STREAM | SOLV_BIN>(a, cfg, s); break;
        case SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN:
            launch_staged<Real, RULE, SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN>(a, cfg, s);
            break;
        default: break;
        }
        return;
    }
    switch (flags) {
    case SOLV_STREAM: launch_direct<Real, RULE, SOLV_STREAM>(a, cfg, s); break;
    case SOLV_BIN: launch_direct<Real, RULE, SOLV_BIN>(a, cfg, s); break;
    case SOLV_COLLIDE: launch_direct<Real, RULE, SOLV_COLLIDE>(a, cfg, s); break;
    case SOLV_STREAM | SOLV_BIN: launch_direct<Real, RULE, SOLV_STREAM | SOLV_BIN>(a, cfg, s); break;
    case SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN:
        launch_direct<Real, RULE, SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN>(a, cfg, s);
        break;
    default: break;
    }
}

void launch_solvent(const StepArgs &a, int flags, LaunchCfg cfg, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    if (a.precision == 1) {
        if (a.rule == 0) dispatch_flags<float, 0>(a, flags, cfg, s);
        else dispatch_flags<float, 1>(a, flags, cfg, s);
    } else {
        if (a.rule == 0) dispatch_flags<double, 0>(a, flags, cfg, s);
        else dispatch_flags<double, 1>(a, flags, cfg, s);
    }
}

size_t solvent_stage_bytes(int precision, int rule, int cap)
{
    if (precision == 1) return rule == 0 ? stage_bytes<float, 0>(cap) : stage_bytes<float, 1>(cap);
    return rule == 0 ? stage_bytes<double, 0>(cap) : stage_bytes<double, 1>(cap);
}

size_t solvent_smem_bytes(int precision, int rule, int cap, int)
{
    return ST_STAGES * solvent_stage_bytes(precision, rule, cap);
}

// ------------------------------------------------------- cell parameters
// Gamma(n/2, 1) variate for n = 3(Nc - 1): floor(n/2) unit exponentials plus
// z^2/2 when n is odd (Eq. 6).  FP32 form: one fast logarithm per pair of
// uniforms (the product of two is >= 2^-66, never subnormal).
__device__ float gamma_half_dof(const DevReplica &r, int64_t step, uint32_t lc, int n_dof, float)
{
    const int nE = n_dof / 2;
    float g = 0.0f;
#pragma unroll 2
    for (int j = 0; 4 * j < nE; ++j) {
        const uint4 w = draw(r, step, lc, TAG_THERMO, (uint32_t)j);
        const int k = nE - 4 * j;
        float p0 = u01f(w.x), p1 = 1.0f;
        if (k > 1) p0 *= u01f(w.y);
        if (k > 2) p1 = u01f(w.z);
        if (k > 3) p1 *= u01f(w.w);
        g -= __logf(p0) + __logf(p1);
    }
    if (n_dof & 1) {
        const uint4 w = draw(r, step, lc, TAG_THERMO_ODD, 0u);
        float sn, cs;
        __sincosf(6.283185307179586f * (u01f(w.y) - 0.5f), &sn, &cs);   // cos(2 pi u) = -cs
        const float z = sqrtf(neg2log(w.x)) * cs;
        g += 0.5f * z * z;
    }
    return g;
}
__device__ double gamma_half_dof(const DevReplica &r, int64_t step, uint32_t lc, int n_dof, double)
{
    int nE = n_dof / 2;
    double g = 0.0;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (int i = 0; i < nE; ++i) {
        if ((i & 3) == 0) w = draw(r, step, lc, TAG_THERMO, (uint32_t)(i >> 2));
        uint32_t x = (i & 3) == 0 ? w.x : (i & 3) == 1 ? w.y : (i & 3) == 2 ? w.z : w.w;
        g += -log(u01d(x));
    }
    if (n_dof & 1) {
        w = draw(r, step, lc, TAG_THERMO_ODD, 0u);
        double z = sqrt(-2.0 * log(u01d(w.x))) * cos(6.283185307179586476925286766559 * u01d(w.y));
        g += 0.5 * z * z;
    }
    return g;
}

// Gamma(a, 1), a = n/2 >= 3/2, by the rejection method of Marsaglia and Tsang
// (ACM Trans. Math. Softw. 26, 363 (2000)): d = a - 1/3, c = 1/sqrt(9 d); a
// standard normal x and a uniform u give v = (1 + c x)^3, accepted (d v) when
// v > 0 and ln u < x^2/2 + d (1 - v + ln v).  Each Philox block (word 3 of the
// counter = block index) gives two attempts: the Box-Muller pair of words 0
// and 1 and the uniforms of words 2 and 3; after MT_MAX_BLOCKS blocks (never
// reached in practice: an attempt is accepted with probability > 0.95) d is
// returned.  FP32 form: the attempt is first tested against the method's
// squeeze u < 1 - 0.0331 x^4, which lies inside the acceptance region, so it
// only decides earlier what the full test would (it holds for ~98 % of the
// attempts and needs no logarithm); otherwise, with y = c x, the full test is
// evaluated as -2 ln u > -x^2 - 2 d (log1p(dv) - dv), dv = v - 1 =
// y (3 + y (3 + y)), which keeps the cancellation of 1 - v + ln v out of it.
// The normals use the fast logarithm (with the complement of u near 1) and
// sine/cosine, whose errors (~1e-6 relative) are far below the tolerance of
// the collision's result.
constexpr uint32_t MT_MAX_BLOCKS = 64;
__device__ float gamma_mt(const DevReplica &r, int64_t step, uint32_t lc, int n_dof, float)
{
    const float a = 0.5f * (float)n_dof;
    const float d = a - 0.333333343f;
    const float c = 1.0f / sqrtf(9.0f * d);
    for (uint32_t k = 0; k < MT_MAX_BLOCKS; ++k) {
        const uint4 w = draw(r, step, lc, TAG_THERMO_MT, k);
        const float rr = sqrtf(neg2log(w.x));
        float sn, cs;
        __sincosf(6.283185307179586f * (u01f(w.y) - 0.5f), &sn, &cs);   // angle shifted by pi
        const float xs[2] = {-rr * cs, -rr * sn};
        const uint32_t us[2] = {w.z, w.w};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float x = xs[j], y = c * x;
            if (y <= -1.0f) continue;
            const float dv = y * (3.0f + y * (3.0f + y));
            const float x2 = x * x;
            if (u01f(us[j]) < 1.0f - 0.0331f * (x2 * x2)) return d * (1.0f + dv);
            if (neg2log(us[j]) > -x2 - 2.0f * d * (log1pf(dv) - dv)) return d * (1.0f + dv);
        }
    }
    return d;
}
__device__ double gamma_mt(const DevReplica &r, int64_t step, uint32_t lc, int n_dof, double)
{
    const double a = 0.5 * (double)n_dof;
    const double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (uint32_t k = 0; k < MT_MAX_BLOCKS; ++k) {
        const uint4 w = draw(r, step, lc, TAG_THERMO_MT, k);
        const double rr = sqrt(-2.0 * log(u01d(w.x)));
        double sn, cs;
        sincos(6.283185307179586476925286766559 * u01d(w.y), &sn, &cs);
        const double xs[2] = {rr * cs, rr * sn};
        const uint32_t us[2] = {w.z, w.w};
        for (int j = 0; j < 2; ++j) {
            const double x = xs[j], t = 1.0 + c * x;
            if (t <= 0.0) continue;
            const double v = t * t * t;
            if (log(u01d(us[j])) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
        }
    }
    return d;
}

// signed 128-bit -> float by magnitude (|error| <= 2 ulp)
__device__ __forceinline__ float i128f(__int128 x)
{
    const bool neg = x < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
    const float f = fmaf(ull2f((unsigned long long)(u >> 64)), 18446744073709551616.0f,
                         ull2f((unsigned long long)u));
    return neg ? -f : f;
}

// Relative kinetic energy E_rel = (S2 - |S1|^2 / M) / 2 of a cell from its exact
// fixed-point sums, rounded once: with S1 in units of 2^-32, S2 of 2^-28 and
// M = Mq 2^-24, 2 M E_rel = 2^-64 X for the integer X = S2 Mq 2^12 - |S1|^2,
// formed exactly in int128 (|X| < 2^127 within the word limits), converted to
// float once and scaled by 2^-65 / M (iM = 1/M).  X < 0 (per-particle roundings of a cell whose members move
// alike) gives 0.
__device__ __forceinline__ float rel_energy_fixed(long long Mq, const long long S1[3], long long S2, float iM)
{
    __int128 X = ((__int128)S2 * Mq) << 12;
#pragma unroll
    for (int k = 0; k < 3; ++k) X -= (__int128)S1[k] * S1[k];
    return fmaxf(i128f(X), 0.0f) * 2.710505431213761085018632e-20f * iM;   // 2^-65 / M
}

// int64 -> float for |w| < 2^48 (a momentum or noise sum), rounded once: the
// magnitude's high 24 and low 24 bits convert exactly and one fused
// multiply-add joins them
__device__ __forceinline__ float ll2f48(long long w)
{
    const unsigned long long m = w < 0 ? 0ull - (unsigned long long)w : (unsigned long long)w;
    const float f = fmaf(__uint2float_rn((uint32_t)(m >> 24)), 16777216.0f, __uint2float_rn((uint32_t)m & 0xFFFFFFu));
    return w < 0 ? -f : f;
}

// FP32 form: cell words -> collision parameters with FP32/integer pipes only.
// Each CTA takes PARAM_TILES consecutive 256-cell tiles, one cell of each per
// thread.  The word loads of all of them are issued before any arithmetic (a
// warp keeps PARAM_TILES x NW loads in flight instead of a chain of dependent
// loads) and parked in shared memory, so the registers of the arithmetic that
// follows are not tied up by the parked words.
constexpr int PARAM_TILES = 2;

template <int RULE>
__device__ __forceinline__ void params32_cell(const StepArgs &a, const DevReplica &r, int64_t step, int64_t c,
                                              const long long (&w)[MAX_WORDS32])
{
    const float kT = a.kTf;
    const float s32 = 2.3283064365386962890625e-10f;   // 2^-32
    long long S1[3], cs, cb;
    unpack48(w[0], cs, S1[0]);
    unpack48(w[1], cb, S1[1]);
    S1[2] = w[2];
    const int ns = (int)cs, nb = (int)cb, n = ns + nb;
    float rec[8] = {0.f, 0.f, 0.f, -1.f, 0.f, 0.f, 0.f, 0.f};
    if (n >= 2) {
        const long long Mq = (long long)ns * a.qm_solvent + (long long)nb * a.qm_site;
        const float M = (float)ns * a.m_solvent_f + (float)nb * a.m_site_f;
        const float iM = 1.0f / M;
        float u[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k] = ll2f48(S1[k]) * s32 * iM;
        rec[0] = u[0]; rec[1] = u[1]; rec[2] = u[2];
        const uint32_t lc = (uint32_t)(c - r.cell_base);
        if (RULE == 0) {
            // axis: z = u1 - (1 - u1), rho = 2 sqrt(u1 (1 - u1)), phi = 2 pi u2
            const uint4 wa = draw(r, step, lc, TAG_AXIS, 0u);
            const float ua = u01f(wa.x), ub = u01f(~wa.x);
            const float zz = ua - ub, rho = 2.0f * sqrtf(ua * ub);
            float sn, cs;
            __sincosf(6.283185307179586f * (u01f(wa.y) - 0.5f), &sn, &cs);   // angle shifted by pi
            rec[4] = -rho * cs; rec[5] = -rho * sn; rec[6] = zz;
            float kappa = 1.0f;
            if (a.thermostat) {
                const float erel = rel_energy_fixed(Mq, S1, w[3], iM);
                const float g = a.thermostat == 2 ? gamma_mt(r, step, lc, 3 * (n - 1), 0.0f)
                                                  : gamma_half_dof(r, step, lc, 3 * (n - 1), 0.0f);
                kappa = erel > 0.0f ? sqrtf(kT * g) * rsqrtf(erel) : 1.0f;
            }
            rec[3] = kappa;
        } else {
            rec[3] = 1.0f;
            rec[4] = ll2f48(w[3]) * s32 * iM; rec[5] = ll2f48(w[4]) * s32 * iM; rec[6] = ll2f48(w[5]) * s32 * iM;
        }
    }
    float4 *o = reinterpret_cast<float4 *>(a.params) + 2 * c;
    o[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
    o[1] = make_float4(rec[4], rec[5], rec[6], 0.0f);
}

template <int RULE>
__global__ void __launch_bounds__(256, 4) k_params32(StepArgs a)
{
    constexpr int NW = Words32<RULE>::n;
    constexpr int K = PARAM_TILES;
    __shared__ long long sw[K][NW][256];
    __shared__ Tile stile[K];
    long long *sums = reinterpret_cast<long long *>(a.sums);
    long long *dbg = reinterpret_cast<long long *>(a.dbg_sums);
    const int64_t C = a.n_cells;
    // CTAs start roughly in index order; they take the cell tiles from the last
    // to the first, so that the words the solvent pass binned last (still in
    // L2) are read first, and the records and cleared words that the next
    // solvent pass (a forward sweep) needs first are the ones written last
    const int t0 = blockIdx.x * K;
    int64_t cell[K];
    int rep[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cell[k] = -1;
        rep[k] = 0;
        if (t0 + k < a.n_ctiles) {
            const Tile tl = a.ctiles[a.n_ctiles - 1 - (t0 + k)];
            const int64_t c = tl.begin + threadIdx.x;
            if (c < tl.end) { cell[k] = c; rep[k] = tl.rep; }
            if (threadIdx.x == 0) stile[k] = tl;
        } else if (threadIdx.x == 0) {
            stile[k] = Tile{0, 0, 0, 0};
        }
    }
    {
        long long w[K][NW];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < NW; ++j) w[k][j] = cell[k] >= 0 ? __ldcs(sums + j * C + cell[k]) : 0ll;
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                sw[k][j][threadIdx.x] = w[k][j];
                if (cell[k] >= 0) {
                    sums[j * C + cell[k]] = 0;
                    if (dbg) dbg[j * C + cell[k]] = w[k][j];
                }
            }
    }
    __syncthreads();   // stile; the words are re-read from shared memory below
    const int64_t step = *a.d_step;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const Tile tl = stile[k];
        const int64_t c = tl.begin + threadIdx.x;
        if (c < tl.end) {
            long long w[MAX_WORDS32] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < NW; ++j) w[j] = sw[k][j][threadIdx.x];
            const DevReplica r = a.reps[tl.rep];
            params32_cell<RULE>(a, r, step, c, w);
        }
    }
}

// FP64 form (plain): the same parameters in double precision
template <typename Real, int RULE>
__global__ void __launch_bounds__(256) k_params(StepArgs a)
{
    constexpr int NW = NWords<Real, RULE>::n;
    typedef typename SumWord<Real>::type W;
    const int64_t step = *a.d_step;
    W *sums = reinterpret_cast<W *>(a.sums);
    W *dbg = reinterpret_cast<W *>(a.dbg_sums);
    const int64_t C = a.n_cells;
    const Real kT = Consts<Real>::kT(a);
    int err = 0;
    for (int t = blockIdx.x; t < a.n_ctiles; t += gridDim.x) {
        const Tile tl = a.ctiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            W w[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                w[k] = sums[k * C + c];
                sums[k * C + c] = W(0);
                if (dbg) dbg[k * C + c] = w[k];
            }
            int n;
            Real M, p[3], s2 = 0, xi[3] = {0, 0, 0};
            {
                n = (int)(double)w[0];
                M = (Real)(double)w[1];
                for (int k = 0; k < 3; ++k) p[k] = (Real)(double)w[2 + k];
                if (RULE == 0) s2 = (Real)(double)w[5];
                else for (int k = 0; k < 3; ++k) xi[k] = (Real)(double)w[5 + k];
            }
            Real rec[8] = {0, 0, 0, Real(-1), 0, 0, 0, 0};
            if (n >= 2) {
                Real u[3] = {p[0] / M, p[1] / M, p[2] / M};
                rec[0] = u[0]; rec[1] = u[1]; rec[2] = u[2];
                const uint32_t lc = (uint32_t)(c - r.cell_base);
                if (RULE == 0) {
                    uint4 wa = draw(r, step, lc, TAG_AXIS, 0u);
                    Real zz, sp, cp;
                    Real rho;
                    {
                        zz = (Real)(2.0 * u01d(wa.x) - 1.0);
                        rho = (Real)sqrt(1.0 - (double)zz * (double)zz);
                        double s_, c_;
                        sincos(6.283185307179586476925286766559 * u01d(wa.y), &s_, &c_);
                        sp = (Real)s_; cp = (Real)c_;
                    }
                    rec[4] = rho * cp; rec[5] = rho * sp; rec[6] = zz;
                    Real kappa = Real(1);
                    if (a.thermostat) {
                        Real erel = Real(0.5) * (s2 - (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) / M);
                        Real g = a.thermostat == 2 ? gamma_mt(r, step, lc, 3 * (n - 1), Real(0))
                                                   : gamma_half_dof(r, step, lc, 3 * (n - 1), Real(0));
                        kappa = erel > Real(0) ? sqrt(kT * g / erel) : Real(1);
                    }
                    rec[3] = kappa;
                } else {
                    rec[3] = Real(1);
                    rec[4] = xi[0] / M; rec[5] = xi[1] / M; rec[6] = xi[2] / M;
                }
            }
            if (sizeof(Real) == 4) {
                float4 *o = reinterpret_cast<float4 *>(a.params) + 2 * c;
                o[0] = make_float4((float)rec[0], (float)rec[1], (float)rec[2], (float)rec[3]);
                o[1] = make_float4((float)rec[4], (float)rec[5], (float)rec[6], 0.0f);
            } else {
                double2 *o = reinterpret_cast<double2 *>(a.params) + 4 * c;
                o[0] = make_double2(rec[0], rec[1]);
                o[1] = make_double2(rec[2], rec[3]);
                o[2] = make_double2(rec[4], rec[5]);
                o[3] = make_double2(rec[6], 0.0);
            }
        }
    }
    if (err) atomicOr(a.d_err, ERR_CELL);
}

void launch_params(const StepArgs &a, int, cudaStream_t s)
{
    if (a.n_ctiles == 0) return;
    const int grid = a.n_ctiles;   // one 256-cell tile per CTA, one cell per thread
    if (a.precision == 1) {
        const int grid32 = (a.n_ctiles + PARAM_TILES - 1) / PARAM_TILES;
        if (a.rule == 0) k_params32<0><<<grid32, 256, 0, s>>>(a);
        else k_params32<1><<<grid32, 256, 0, s>>>(a);
    } else {
        if (a.rule == 0) k_params<double, 0><<<grid, 256, 0, s>>>(a);
        else k_params<double, 1><<<grid, 256, 0, s>>>(a);
    }
}

// ------------------------------------------------- layout transforms (I/O)
// host rows (tag order) -> SoA slots; positions outside [0, L) set ERR_POSITION
template <typename Real>
__global__ void k_aos_to_soa(StepArgs a, const Real *xa, const Real *va)
{
    Real *X[3] = {(Real *)a.x, (Real *)a.y, (Real *)a.z};
    Real *V[3] = {(Real *)a.vx, (Real *)a.vy, (Real *)a.vz};
    int bad = 0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            int64_t tag = i - r.solv_begin, row = r.row_begin + tag;
            for (int k = 0; k < 3; ++k) {
                Real x = xa[3 * row + k];
                bad |= !(x >= Real(0) && x < (Real)r.L[k]);
                X[k][i] = x;
                V[k][i] = va[3 * row + k];
            }
            a.tag[i] = (uint32_t)tag;
        }
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

template <typename Real>
__global__ void k_soa_to_aos(StepArgs a, Real *xa, Real *va)
{
    const Real *X[3] = {(const Real *)a.x, (const Real *)a.y, (const Real *)a.z};
    const Real *V[3] = {(const Real *)a.vx, (const Real *)a.vy, (const Real *)a.vz};
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            uint32_t tag = a.tag[i];
            if (tag == PAD_TAG || (int64_t)tag >= r.n_solvent) continue;
            int64_t row = r.row_begin + tag;
            for (int k = 0; k < 3; ++k) {
                xa[3 * row + k] = X[k][i];
                va[3 * row + k] = V[k][i];
            }
        }
    }
}

void launch_aos_to_soa(const StepArgs &a, const void *xaos, const void *vaos, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    if (a.precision == 1) k_aos_to_soa<float><<<a.n_tiles, 256, 0, s>>>(a, (const float *)xaos, (const float *)vaos);
    else k_aos_to_soa<double><<<a.n_tiles, 256, 0, s>>>(a, (const double *)xaos, (const double *)vaos);
}

void launch_soa_to_aos(const StepArgs &a, void *xaos, void *vaos, const int64_t *, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    if (a.precision == 1) k_soa_to_aos<float><<<a.n_tiles, 256, 0, s>>>(a, (float *)xaos, (float *)vaos);
    else k_soa_to_aos<double><<<a.n_tiles, 256, 0, s>>>(a, (double *)xaos, (double *)vaos);
}

// ---------------------------------------------------- FP64 diagnostics
template <typename Real>
__global__ void k_solvent_diag(StepArgs a, double *acc)
{
    const Real *V[3] = {(const Real *)a.vx, (const Real *)a.vy, (const Real *)a.vz};
    double s[4] = {0, 0, 0, 0};
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            double vx = (double)V[0][i], vy = (double)V[1][i], vz = (double)V[2][i];
            s[0] += vx; s[1] += vy; s[2] += vz;
            s[3] += vx * vx + vy * vy + vz * vz;
        }
    }
    for (int k = 0; k < 4; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, v);
    }
}

void launch_solvent_diag(const StepArgs &a, double *acc, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    int grid = a.n_tiles < 1024 ? a.n_tiles : 1024;
    if (a.precision == 1) k_solvent_diag<float><<<grid, 256, 0, s>>>(a, acc);
    else k_solvent_diag<double><<<grid, 256, 0, s>>>(a, acc);
}

// ------------------------------------------------------------- re-sort
template <typename Real>
__device__ __forceinline__ int plain_cell(const DevReplica &r, Real x, Real y, Real z)
{
    return r.cell_base + cell_axis(x, 0, r.L[0]) +
           r.L[0] * (cell_axis(y, 0, r.L[1]) + r.L[1] * cell_axis(z, 0, r.L[2]));
}

// four consecutive elements from i (a multiple of 4 inside a tile that starts
// on an 8-element boundary): one vector load when all four are in the tile
__device__ __forceinline__ void load4_tail(const float *p, int64_t i, int64_t end, float (&o)[4])
{
    if (i + 4 <= end) {
        const float4 t = *reinterpret_cast<const float4 *>(p + i);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = i + j < end ? p[i + j] : 0.0f;
    }
}
__device__ __forceinline__ void load4_tail(const double *p, int64_t i, int64_t end, double (&o)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = i + j < end ? p[i + j] : 0.0;
}

// histogram of the cells (four particles per thread, 1024-particle units of
// the state-transfer tiles)
template <typename Real>
__global__ void __launch_bounds__(256) k_sort_count(StepArgs a, int32_t *counts)
{
    const Real *X = (const Real *)a.x, *Y = (const Real *)a.y, *Z = (const Real *)a.z;
    const int units = a.n_tiles * (2048 / 1024);
    for (int w = blockIdx.x; w < units; w += gridDim.x) {
        const Tile tl = a.tiles[w >> 1];
        const DevReplica r = a.reps[tl.rep];
        const int64_t i0 = tl.begin + (int64_t)(w & 1) * 1024 + 4 * threadIdx.x;
        if (i0 >= tl.end) continue;
        Real x[4], y[4], z[4];
        load4_tail(X, i0, tl.end, x);
        load4_tail(Y, i0, tl.end, y);
        load4_tail(Z, i0, tl.end, z);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i0 + j < tl.end) atomicAdd(counts + plain_cell(r, x[j], y[j], z[j]), 1);
    }
}

void launch_sort_count(const StepArgs &a, int32_t *counts, int num_sms, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    const int grid = std::min(2 * a.n_tiles, num_sms * 8);
    if (a.precision == 1) k_sort_count<float><<<grid, 256, 0, s>>>(a, counts);
    else k_sort_count<double><<<grid, 256, 0, s>>>(a, counts);
}

// exclusive scan: chunks of SCAN_CHUNK elements, one CTA of 1024 threads per chunk
constexpr int SCAN_THREADS = 1024, SCAN_ITEMS = 8, SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

size_t scan_block_sums_size(int64_t n) { return (size_t)((n + SCAN_CHUNK - 1) / SCAN_CHUNK) + 1; }

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *sh, int32_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int32_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t *in, int64_t n, int32_t *bs)
{
    __shared__ int32_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) v += in[base + k];
    int32_t total;
    block_exclusive_scan(v, sh, total);
    if (threadIdx.x == 0) bs[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_blocks(int32_t *bs, int64_t nb)
{
    // exclusive scan of the chunk totals, in passes of SCAN_CHUNK
    __shared__ int32_t sh[32];
    int32_t carry = 0;
    for (int64_t off = 0; off < nb; off += SCAN_CHUNK) {
        int64_t base = off + (int64_t)threadIdx.x * SCAN_ITEMS;
        int32_t loc[SCAN_ITEMS];
        int32_t v = 0;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            loc[k] = (base + k < nb) ? bs[base + k] : 0;
            v += loc[k];
        }
        int32_t total;
        int32_t ex = block_exclusive_scan(v, sh, total) + carry;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < nb) bs[base + k] = ex;
            ex += loc[k];
        }
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_final(const int32_t *in, int32_t *out, int64_t n,
                                                            const int32_t *bs)
{
    __shared__ int32_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t loc[SCAN_ITEMS];
    int32_t v = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = (base + k < n) ? in[base + k] : 0;
        v += loc[k];
    }
    int32_t total;
    int32_t ex = block_exclusive_scan(v, sh, total) + bs[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += loc[k];
    }
}

void launch_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *bs, cudaStream_t s)
{
    if (n <= 0) return;
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bs);
    k_scan_blocks<<<1, SCAN_THREADS, 0, s>>>(bs, nb);
    k_scan_final<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, bs);
}

// Re-sort by rank and gather.  A scatter of the six state arrays and the tags
// writes each destination sector in pieces (the particles of one cell arrive
// from different places of the source order, at different times), and the
// pieces that leave L2 before their sector is complete cost a read-modify-write
// in DRAM.  Instead the rank pass scatters only one 4-byte source index per
// particle; the gather pass then writes every destination array in order and
// reads the sources, which lie close together (the state was cell-sorted a few
// steps earlier), mostly from L2.
//
// Both passes take 1024-element units of the state-transfer tiles round robin
// over the grid (four consecutive elements per thread, whose memory accesses
// are independent and overlap), so that the CTAs in flight cover one compact
// window of the state (about grid x 1024 elements) and the sources that
// neighbouring destinations share are still in L2 when they are read again.
constexpr int SORT_UNIT = 1024, SORT_UNITS = 2048 / SORT_UNIT;   // units per state-transfer tile
#ifndef GATHER_CTAS_PER_SM
#define GATHER_CTAS_PER_SM 4
#endif

// rank: destination slot = the cell's first slot + a cursor; the lanes of a
// warp in one cell take consecutive slots with one atomic.  perm[slot] = the
// particle's row in its replica.  Lane l of a warp takes particles 32 j + l of
// the warp's 128 (j = 0..3), so that each warp-wide match covers 32 consecutive
// particles of the sorted source, which fall into few cells (at L=200: 1.90
// against 2.15 ms per re-sort, together with the same layout in the gather).
// SHIFTED: the cells are those of the next collision (the grid shift of step
// *d_step + 1, the binning rule of the solvent pass), whose solvent counts the
// cell words already hold; else the unshifted cells.
template <typename Real, bool SHIFTED>
__global__ void __launch_bounds__(256) k_sort_rank(StepArgs a, const int32_t *ex, const int32_t *counts,
                                                   int32_t *cursor, uint32_t *perm)
{
    const Real *X = (const Real *)a.x, *Y = (const Real *)a.y, *Z = (const Real *)a.z;
    const unsigned lane = threadIdx.x & 31u;
    const int units = a.n_tiles * SORT_UNITS;
    const int64_t step1 = *a.d_step + 1;
    int last_rep = -1;
    typename ShiftT<Real>::type sh[3] = {};
    for (int w = blockIdx.x; w < units; w += gridDim.x) {   // uniform trip count (warp votes)
        const Tile tl = a.tiles[w / SORT_UNITS];
        const DevReplica r = a.reps[tl.rep];
        if (SHIFTED && tl.rep != last_rep) {
            int32_t S[3];
            grid_shift(r, step1, S);
            for (int k = 0; k < 3; ++k) sh[k] = shift_as(S[k], typename ShiftT<Real>::type());
            last_rep = tl.rep;
        }
        // lane l of warp k takes particles u0 + 32 j (j = 0..3) of the unit: each j
        // covers 32 consecutive particles, so a warp's atomics per cell are fewer
        const int64_t u0 = tl.begin + (int64_t)(w % SORT_UNITS) * SORT_UNIT + 128 * (threadIdx.x >> 5) + lane;
        int c[4], base[4];
        bool v[4];
        unsigned peers[4];
        Real x[4], y[4], z[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = u0 + 32 * j;
            const bool in = i < tl.end;
            x[j] = in ? X[i] : Real(0);
            y[j] = in ? Y[i] : Real(0);
            z[j] = in ? Z[i] : Real(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = u0 + 32 * j < tl.end;
            if (SHIFTED)
                c[j] = v[j] ? r.cell_base + cell_bin(x[j], sh[0], r.L[0]) +
                                  r.L[0] * (cell_bin(y[j], sh[1], r.L[1]) + r.L[1] * cell_bin(z[j], sh[2], r.L[2]))
                            : 0;
            else
                c[j] = v[j] ? plain_cell(r, x[j], y[j], z[j]) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned act = __ballot_sync(0xffffffffu, v[j]);
            peers[j] = v[j] ? __match_any_sync(act, c[j]) : 0u;
            base[j] = 0;
        }
        // the cells' offsets and counts are read before the atomics (whose
        // returns the loads could not pass), and the leaders' atomics are
        // independent: all of them are in flight together
        const int32_t ex0 = ex[r.cell_base];
        int32_t off[4], cnt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            off[j] = v[j] ? ex[c[j]] - ex0 : 0;
            cnt[j] = v[j] ? counts[c[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (v[j] && (int)lane == __ffs(peers[j]) - 1) base[j] = atomicAdd(cursor + c[j], __popc(peers[j]));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned act = __ballot_sync(0xffffffffu, v[j]);
            if (v[j]) {
                const int b = __shfl_sync(act, base[j], __ffs(peers[j]) - 1) + __popc(peers[j] & ((1u << lane) - 1u));
                if (b < cnt[j]) {
                    perm[r.solv_begin + off[j] + b] = (uint32_t)(u0 + 32 * j - r.solv_begin);
                } else {   // more particles than the cell's count: no access
                    atomicOr(a.d_err, ERR_INDEX);
                    atomicCAS(a.d_err + 1, 0, 7);
                }
            }
        }
    }
}

// gather: every slot of the replica reads its particle's arrays and tag
template <typename Real>
__global__ void __launch_bounds__(256) k_sort_gather(StepArgs a, const uint32_t *perm, Real *d0, Real *d1, Real *d2,
                                                    Real *d3, Real *d4, Real *d5, uint32_t *dtag)
{
    const Real *S[6] = {(const Real *)a.x, (const Real *)a.y, (const Real *)a.z,
                        (const Real *)a.vx, (const Real *)a.vy, (const Real *)a.vz};
    Real *D[6] = {d0, d1, d2, d3, d4, d5};
    const int units = a.n_tiles * SORT_UNITS;
    for (int w = blockIdx.x; w < units; w += gridDim.x) {
        const Tile tl = a.tiles[w / SORT_UNITS];
        const DevReplica r = a.reps[tl.rep];
        // lane l of warp k fills slots u0 + 32 j (j = 0..3) of the unit
        const int64_t u0 = tl.begin + (int64_t)(w % SORT_UNITS) * SORT_UNIT + 128 * (threadIdx.x >> 5) +
                           (threadIdx.x & 31);
        if (u0 >= tl.end) continue;
        int64_t src[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t d = u0 + 32 * j;
            const bool in = d < tl.end;
            const uint32_t q = in ? perm[d] : 0u;
            ok[j] = in && (int64_t)q < r.n_solvent;
            if (in && !ok[j]) {   // a slot no particle was ranked into: no access
                atomicOr(a.d_err, ERR_INDEX);
                atomicCAS(a.d_err + 1, 0, 6);
            }
            src[j] = r.solv_begin + (ok[j] ? q : 0u);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            Real o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = S[k][src[j]];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j]) D[k][u0 + 32 * j] = o[j];
        }
        uint32_t tg[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tg[j] = a.tag[src[j]];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) dtag[u0 + 32 * j] = tg[j];
    }
}

// solvent counts of the next collision's cells from the cell words (FP32 form:
// the high 16 bits of word 0 with the signed low 48 bits taken off)
__global__ void k_counts_from_words(int64_t C, const long long *w0, int32_t *counts)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        long long n, lo;
        unpack48(w0[c], n, lo);
        counts[c] = (int32_t)n;
    }
}

void launch_counts_from_words(int64_t C, const void *sums, int32_t *counts, int num_sms, cudaStream_t s)
{
    if (C == 0) return;
    k_counts_from_words<<<num_sms * 8, 256, 0, s>>>(C, reinterpret_cast<const long long *>(sums), counts);
}

void launch_sort_rank_gather(const StepArgs &a, const int32_t *ex, const int32_t *counts, int32_t *cursor,
                             uint32_t *perm, void *const d[6], uint32_t *dtag, bool shifted, int num_sms,
                             cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    // rank: full occupancy (its atomics' round trips need many warps); gather:
    // GATHER_CTAS_PER_SM CTAs per SM, so that its window of the state stays in L2
    const int units = a.n_tiles * SORT_UNITS;
    const int grid_r = std::min(units, num_sms * 8), grid_g = std::min(units, num_sms * GATHER_CTAS_PER_SM);
    if (a.precision == 1) {
        if (shifted) k_sort_rank<float, true><<<grid_r, 256, 0, s>>>(a, ex, counts, cursor, perm);
        else k_sort_rank<float, false><<<grid_r, 256, 0, s>>>(a, ex, counts, cursor, perm);
        k_sort_gather<float><<<grid_g, 256, 0, s>>>(a, perm, (float *)d[0], (float *)d[1], (float *)d[2],
                                                    (float *)d[3], (float *)d[4], (float *)d[5], dtag);
    } else {
        k_sort_rank<double, false><<<grid_r, 256, 0, s>>>(a, ex, counts, cursor, perm);   // counts by the count pass
        k_sort_gather<double><<<grid_g, 256, 0, s>>>(a, perm, (double *)d[0], (double *)d[1], (double *)d[2],
                                                     (double *)d[3], (double *)d[4], (double *)d[5], dtag);
    }
}

// order every cell's segment by tag (insertion sort; segments hold ~10)
template <typename Real>
__global__ void k_sort_canonical(StepArgs a, Real *d0, Real *d1, Real *d2, Real *d3, Real *d4, Real *d5,
                                 uint32_t *tag, const int32_t *ex)
{
    Real *D[6] = {d0, d1, d2, d3, d4, d5};
    for (int t = blockIdx.x; t < a.n_ctiles; t += gridDim.x) {
        const Tile tl = a.ctiles[t];
        const DevReplica r = a.reps[tl.rep];
        const int32_t ex0 = ex[r.cell_base];
        const int64_t cend = (int64_t)r.cell_base + (int64_t)r.L[0] * r.L[1] * r.L[2];
        for (int64_t c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            int64_t b = r.solv_begin + (ex[c] - ex0);
            int64_t e = r.solv_begin + ((c + 1 < cend ? ex[c + 1] : ex0 + (int32_t)r.n_solvent) - ex0);
            for (int64_t i = b + 1; i < e; ++i) {
                uint32_t key = tag[i];
                Real v[6];
                for (int k = 0; k < 6; ++k) v[k] = D[k][i];
                int64_t j = i - 1;
                while (j >= b && tag[j] > key) {
                    tag[j + 1] = tag[j];
                    for (int k = 0; k < 6; ++k) D[k][j + 1] = D[k][j];
                    --j;
                }
                tag[j + 1] = key;
                for (int k = 0; k < 6; ++k) D[k][j + 1] = v[k];
            }
        }
    }
}

void launch_sort_canonical(const StepArgs &a, void *const d[6], uint32_t *tag, const int32_t *ex,
                           cudaStream_t s)
{
    if (a.n_ctiles == 0) return;
    if (a.precision == 1)
        k_sort_canonical<float><<<a.n_ctiles, 256, 0, s>>>(a, (float *)d[0], (float *)d[1], (float *)d[2],
                                                          (float *)d[3], (float *)d[4], (float *)d[5], tag, ex);
    else
        k_sort_canonical<double><<<a.n_ctiles, 256, 0, s>>>(a, (double *)d[0], (double *)d[1], (double *)d[2],
                                                           (double *)d[3], (double *)d[4], (double *)d[5], tag,
                                                           ex);
}


// ------------------------------------------ RNEMD exchange (Sec. III.B)
// Reverse non-equilibrium (Mueller-Plathe) exchange of v_x between the solvent
// particles of slab A closest to +v_t and those of slab B closest to -v_t.
// Three launches.  k_rnemd_scan reads y of every particle (vector loads) and
// v_x of the slab members only; it lists the members with their rank keys
// (each CTA gathers its members in shared memory and reserves global space
// once) and histograms the keys per slab in 1/8-octave buckets.
// k_rnemd_filter finds, in every CTA, the bucket holding the max_pairs-th
// smallest key of each slab and keeps the listed members up to it as
// candidates.  k_rnemd_select, one CTA, sorts the candidates (key, then id) and
// exchanges the pairs.  When the solvent is already binned for the coming collision the
// exchanged particles' contributions to the cell words are corrected exactly
// (the difference of their old and new terms).
// 1/8-octave bucket of a non-negative key (float bits >> 20), clamped to the
// RN_BUCKETS buckets that start at 2^-40: monotone in the key
__device__ __forceinline__ int rn_bucket(float k)
{
    constexpr int lo = (127 - 40) << 3;   // bucket of 2^-40
    return min(max((int)(__float_as_uint(k) >> 20) - lo, 0), RN_BUCKETS - 1);
}
__device__ __forceinline__ unsigned long long rn_bits(float k) { return (unsigned long long)__float_as_uint(k); }
__device__ __forceinline__ unsigned long long rn_bits(double k)
{
    return (unsigned long long)__double_as_longlong(k);
}
template <typename Real> __device__ __forceinline__ int rn_bucket_of_bits(unsigned long long b);
template <> __device__ __forceinline__ int rn_bucket_of_bits<float>(unsigned long long b)
{
    return rn_bucket(__uint_as_float((uint32_t)b));
}
template <> __device__ __forceinline__ int rn_bucket_of_bits<double>(unsigned long long b)
{
    return rn_bucket((float)__longlong_as_double((long long)b));
}
__device__ __forceinline__ int rn_slab(const RnemdArgs &g, float y)
{
    return (y >= g.ya0f && y < g.ya1f) ? 0 : (y >= g.yb0f && y < g.yb1f) ? 1 : -1;
}
__device__ __forceinline__ int rn_slab(const RnemdArgs &g, double y)
{
    return (y >= g.ya0 && y < g.ya1) ? 0 : (y >= g.yb0 && y < g.yb1) ? 1 : -1;
}
__device__ __forceinline__ float rn_key(const RnemdArgs &g, float vx, int slab)
{
    return fabsf(slab == 0 ? __fsub_rn(vx, g.vtf) : __fadd_rn(vx, g.vtf));
}
__device__ __forceinline__ double rn_key(const RnemdArgs &g, double vx, int slab)
{
    return fabs(slab == 0 ? __dsub_rn(vx, g.vt) : __dadd_rn(vx, g.vt));
}
__device__ __forceinline__ bool rn_due(const StepArgs &a, const RnemdArgs &g)
{
    return (*a.d_step + g.step_offset) % g.period == 0;
}

// members a CTA gathers in shared memory per slab; the launcher sizes the grid
// so that a CTA's share of a slab fits (the rest would go one by one to the
// global list through contended atomics)
constexpr int RN_SBUF = 512;

template <typename Real>
__global__ void __launch_bounds__(512) k_rnemd_scan(StepArgs a, RnemdArgs g)
{
    __shared__ int sh[2 * RN_BUCKETS];
    __shared__ RnEntry sbuf[2][RN_SBUF];
    __shared__ int scount[2], sbase[2];
    if (!rn_due(a, g)) return;
    for (int b = threadIdx.x; b < 2 * RN_BUCKETS; b += blockDim.x) sh[b] = 0;
    if (threadIdx.x < 2) scount[threadIdx.x] = 0;
    __syncthreads();
    const DevReplica r = a.reps[0];
    const Real *Y = (const Real *)a.y, *VX = (const Real *)a.vx;
    const int64_t beg = r.solv_begin, n = r.n_solvent;
    int bad = 0;
    auto visit = [&](int64_t i, Real y) {
        const int sl = rn_slab(g, y);
        if (sl < 0) return;
        const Real k = rn_key(g, VX[beg + i], sl);
        atomicAdd(&sh[sl * RN_BUCKETS + rn_bucket((float)k)], 1);
        const RnEntry e{rn_bits(k), a.tag[beg + i], (uint32_t)i};
        const int pos = atomicAdd(&scount[sl], 1);
        if (pos < RN_SBUF) {
            sbuf[sl][pos] = e;
        } else {   // a crowded CTA: straight to the global list
            const int gp = atomicAdd(&g.count[sl], 1);
            if (gp < RN_LIST) g.list[(int64_t)sl * RN_LIST + gp] = e;
            else bad = 1;
        }
    };
    // four consecutive particles per vector load of y (the replica's first
    // slot is a multiple of 8), RN_LOADS loads in flight per thread: the pass
    // is bound by how many bytes are in flight
    constexpr int RN_LOADS = 4;
    const int64_t n4 = n & ~(int64_t)3;
    const int64_t stride = 4 * (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); i < n4; i += RN_LOADS * stride) {
        Real y[RN_LOADS][4];
#pragma unroll
        for (int u = 0; u < RN_LOADS; ++u)
            if (i + u * stride < n4) ld4(Y + beg + i + u * stride, y[u]);
#pragma unroll
        for (int u = 0; u < RN_LOADS; ++u)
            if (i + u * stride < n4)
#pragma unroll
                for (int j = 0; j < 4; ++j) visit(i + u * stride + j, y[u][j]);
    }
    if (blockIdx.x == 0 && threadIdx.x < n - n4) visit(n4 + threadIdx.x, Y[beg + n4 + threadIdx.x]);
    __syncthreads();
    if (threadIdx.x < 2) {
        const int m = min(scount[threadIdx.x], RN_SBUF);
        sbase[threadIdx.x] = m ? atomicAdd(&g.count[threadIdx.x], m) : 0;
    }
    __syncthreads();
    for (int sl = 0; sl < 2; ++sl) {
        const int m = min(scount[sl], RN_SBUF);
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const int gp = sbase[sl] + j;
            if (gp < RN_LIST) g.list[(int64_t)sl * RN_LIST + gp] = sbuf[sl][j];
            else bad = 1;
        }
    }
    for (int b = threadIdx.x; b < 2 * RN_BUCKETS; b += blockDim.x)
        if (sh[b]) atomicAdd(&g.hist[b], sh[b]);
    if (bad) atomicOr(a.d_err, ERR_RNEMD);
}

__device__ __forceinline__ bool rn_less(const RnEntry &p, const RnEntry &q)
{
    return p.key < q.key || (p.key == q.key && p.tag < q.tag);
}

// exact change of one particle's cell words when its v_x changes from v0 to v1
template <int RULE>
__device__ __forceinline__ void rn_fix(const StepArgs &a, int c, float v0, float v1, float vy, float vz)
{
    constexpr int NW = Words32<RULE>::n;
    const float xi[3] = {0.f, 0.f, 0.f};
    long long w0[MAX_WORDS32], w1[MAX_WORDS32];
    record_terms<RULE>(a.m_solvent_f, v0, vy, vz, xi, false, w0);
    record_terms<RULE>(a.m_solvent_f, v1, vy, vz, xi, false, w1);
    long long *sums = reinterpret_cast<long long *>(a.sums);
#pragma unroll
    for (int k = 0; k < NW; ++k)
        if (w1[k] != w0[k]) red_add(sums + k * a.n_cells + c, w1[k] - w0[k]);
}
template <int RULE>
__device__ __forceinline__ void rn_fix(const StepArgs &a, int c, double v0, double v1, double vy, double vz)
{
    constexpr int NW = RULE == 0 ? 6 : 8;
    const double xi[3] = {0.0, 0.0, 0.0};
    double w0[NW], w1[NW];
    terms64<RULE>(a.m_solvent, v0, vy, vz, xi, w0);
    terms64<RULE>(a.m_solvent, v1, vy, vz, xi, w1);
    double *sums = reinterpret_cast<double *>(a.sums);
#pragma unroll
    for (int k = 0; k < NW; ++k)
        if (w1[k] != w0[k]) red_add(sums + k * a.n_cells + c, w1[k] - w0[k]);
}

// threshold bucket of slab w (computed by warp w of the CTA): the first bucket
// at which the running count reaches max_pairs (every bucket if the slab holds
// fewer; none for max_pairs = 0)
__device__ __forceinline__ int rn_threshold(const RnemdArgs &g, int w)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    constexpr int PER = RN_BUCKETS / 32;
    const int *h = g.hist + w * RN_BUCKETS;
    int part = 0;
    for (int j = 0; j < PER; ++j) part += h[lane * PER + j];
    int incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int before = incl - part, total = __shfl_sync(FULL, incl, 31);
    if (g.max_pairs == 0) return -1;
    if (total <= g.max_pairs) return RN_BUCKETS - 1;
    const unsigned hit = __ballot_sync(FULL, before < g.max_pairs && incl >= g.max_pairs);
    const int owner = __ffs(hit) - 1;
    int tb = 0;
    if (lane == owner) {
        int cum = before;
        for (int j = 0; j < PER; ++j) {
            cum += h[lane * PER + j];
            if (cum >= g.max_pairs) { tb = lane * PER + j; break; }
        }
    }
    return __shfl_sync(FULL, tb, owner);
}

template <typename Real>
__global__ void __launch_bounds__(512) k_rnemd_filter(StepArgs a, RnemdArgs g)
{
    __shared__ int thr[2];
    if (!rn_due(a, g)) return;
    const int warp = threadIdx.x >> 5;
    if (warp < 2) {
        const int t = rn_threshold(g, warp);
        if ((threadIdx.x & 31) == 0) thr[warp] = t;
    }
    __syncthreads();
    for (int sl = 0; sl < 2; ++sl) {
        const int n = min(g.count[sl], RN_LIST);
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
            const RnEntry e = g.list[(int64_t)sl * RN_LIST + j];
            if (rn_bucket_of_bits<Real>(e.key) > thr[sl]) continue;
            const int pos = atomicAdd(&g.ncand[sl], 1);
            if (pos < RN_CAP) g.cand[sl * RN_CAP + pos] = e;
        }
    }
}

template <typename Real, int RULE>
__global__ void __launch_bounds__(1024) k_rnemd_select(StepArgs a, RnemdArgs g)
{
    extern __shared__ __align__(16) unsigned char rn_smem[];
    RnEntry *E = reinterpret_cast<RnEntry *>(rn_smem);   // [2][RN_CAP]
    __shared__ double red[32];
    if (!rn_due(a, g)) return;
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool listed = g.count[0] <= RN_LIST && g.count[1] <= RN_LIST;
    const int nA = g.ncand[0], nB = g.ncand[1];
    if (listed && nA <= RN_CAP && nB <= RN_CAP) {
        for (int t = threadIdx.x; t < nA; t += blockDim.x) E[t] = g.cand[t];
        for (int t = threadIdx.x; t < nB; t += blockDim.x) E[RN_CAP + t] = g.cand[RN_CAP + t];
    }
    if (!listed || nA > RN_CAP || nB > RN_CAP) {
        if (threadIdx.x == 0) atomicOr(a.d_err, ERR_RNEMD);
    } else {
        int P = 2;
        while (P < nA || P < nB) P <<= 1;
        const RnEntry pad{~0ull, ~0u, 0u};
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
            if (t >= nA) E[t] = pad;
            if (t >= nB) E[RN_CAP + t] = pad;
        }
        __syncthreads();
        // bitonic sort of both lists, ascending by (key, id)
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < 2 * P; t += blockDim.x) {
                    const int l = t >= P ? 1 : 0, u = t - l * P, v = u ^ j;
                    if (v > u) {
                        RnEntry &p = E[l * RN_CAP + u], &q = E[l * RN_CAP + v];
                        const bool up = (u & k) == 0;
                        if (rn_less(q, p) == up) {
                            const RnEntry w = p;
                            p = q;
                            q = w;
                        }
                    }
                }
                __syncthreads();
            }
        const int np = min(g.max_pairs, min(nA, nB));
        const DevReplica r = a.reps[0];
        Real *X = (Real *)a.x, *Y = (Real *)a.y, *Z = (Real *)a.z;
        Real *VX = (Real *)a.vx, *VY = (Real *)a.vy, *VZ = (Real *)a.vz;
        int32_t S[3] = {0, 0, 0};
        if (g.fix_sums) grid_shift(r, *a.d_step + g.step_offset, S);
        double dp = 0.0;
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const int64_t ia = r.solv_begin + E[i].idx, ib = r.solv_begin + E[RN_CAP + i].idx;
            const Real va = VX[ia], vb = VX[ib];
            VX[ia] = vb;
            VX[ib] = va;
            dp += (double)Consts<Real>::m(a) * ((double)va - (double)vb);
            if (g.fix_sums) {
                const int ca = r.cell_base + cell_axis(X[ia], S[0], r.L[0]) +
                               r.L[0] * (cell_axis(Y[ia], S[1], r.L[1]) + r.L[1] * cell_axis(Z[ia], S[2], r.L[2]));
                const int cb = r.cell_base + cell_axis(X[ib], S[0], r.L[0]) +
                               r.L[0] * (cell_axis(Y[ib], S[1], r.L[1]) + r.L[1] * cell_axis(Z[ib], S[2], r.L[2]));
                rn_fix<RULE>(a, ca, va, vb, VY[ia], VZ[ia]);
                rn_fix<RULE>(a, cb, vb, va, VY[ib], VZ[ib]);
            }
        }
        // deterministic block sum of the exchanged momentum
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dp += __shfl_down_sync(FULL, dp, o);
        if (lane == 0) red[warp] = dp;
        __syncthreads();
        if (warp == 0) {
            double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
            if (lane == 0) {
                *g.p_total += v;
                *g.n_total += np;
            }
        }
    }
    // ready for the next exchange
    for (int b = threadIdx.x; b < 2 * RN_BUCKETS; b += blockDim.x) g.hist[b] = 0;
    if (threadIdx.x < 2) {
        g.count[threadIdx.x] = 0;
        g.ncand[threadIdx.x] = 0;
    }
}

size_t rnemd_swap_smem() { return (size_t)2 * RN_CAP * sizeof(RnEntry); }

template <typename Real, int RULE>
static void launch_rnemd_t(const StepArgs &a, const RnemdArgs &g, int num_sms, int64_t slab_members,
                           cudaStream_t s)
{
    smem_opt_in((const void *)k_rnemd_select<Real, RULE>, rnemd_swap_smem());
    const int64_t want = (3 * slab_members / 2 + RN_SBUF - 1) / RN_SBUF;   // 50 % margin
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(3 * (int64_t)num_sms, want), 1 << 20);
    k_rnemd_scan<Real><<<grid, 512, 0, s>>>(a, g);
    k_rnemd_filter<Real><<<std::max(1, num_sms), 512, 0, s>>>(a, g);
    k_rnemd_select<Real, RULE><<<1, 1024, rnemd_swap_smem(), s>>>(a, g);
}

void launch_rnemd(const StepArgs &a, const RnemdArgs &g, int num_sms, int64_t slab_members, cudaStream_t s)
{
    if (a.precision == 1) {
        if (a.rule == 0) launch_rnemd_t<float, 0>(a, g, num_sms, slab_members, s);
        else launch_rnemd_t<float, 1>(a, g, num_sms, slab_members, s);
    } else {
        if (a.rule == 0) launch_rnemd_t<double, 0>(a, g, num_sms, slab_members, s);
        else launch_rnemd_t<double, 1>(a, g, num_sms, slab_members, s);
    }
}

// ------------------------------------------ velocity profile (Sec. III.B)
constexpr int PROFILE_MAX_BINS = 2048;

template <typename Real>
__global__ void __launch_bounds__(512) k_velocity_profile(StepArgs a, int bin_axis, int vel_axis, int n_bins,
                                                          double *mass, double *mom)
{
    __shared__ double sm[2 * PROFILE_MAX_BINS];
    for (int b = threadIdx.x; b < 2 * n_bins; b += blockDim.x) sm[b] = 0.0;
    __syncthreads();
    const DevReplica r = a.reps[0];
    const Real *B = (const Real *)(bin_axis == 0 ? a.x : bin_axis == 1 ? a.y : a.z);
    const Real *V = (const Real *)(vel_axis == 0 ? a.vx : vel_axis == 1 ? a.vy : a.vz);
    const double scale = (double)n_bins / (double)r.L[bin_axis];
    const double m = a.m_solvent;
    const int64_t end = r.solv_begin + r.n_solvent;
    for (int64_t i = r.solv_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = min(n_bins - 1, max(0, (int)floor((double)B[i] * scale)));
        atomicAdd(&sm[b], m);
        atomicAdd(&sm[n_bins + b], m * (double)V[i]);
    }
    if (blockIdx.x == 0)
        for (int64_t j = r.body_begin + threadIdx.x; j < r.body_end; j += blockDim.x) {
            const DevBody &bd = a.bodies[j];
            const int b = min(n_bins - 1, max(0, (int)floor(bd.R[bin_axis] * scale)));
            atomicAdd(&sm[b], a.shapes[bd.shape].M);
            atomicAdd(&sm[n_bins + b], bd.P[vel_axis]);
        }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        if (sm[b] != 0.0) atomicAdd(&mass[b], sm[b]);
        if (sm[n_bins + b] != 0.0) atomicAdd(&mom[b], sm[n_bins + b]);
    }
}

void launch_velocity_profile(const StepArgs &a, int bin_axis, int vel_axis, int n_bins, double *mass, double *mom,
                             int num_sms, cudaStream_t s)
{
    const int grid = std::max(1, num_sms);
    if (a.precision == 1) k_velocity_profile<float><<<grid, 512, 0, s>>>(a, bin_axis, vel_axis, n_bins, mass, mom);
    else k_velocity_profile<double><<<grid, 512, 0, s>>>(a, bin_axis, vel_axis, n_bins, mass, mom);
}


// ------------------------------------- canonical member order (Sec. II.A)
// The binning step as a counting sort: every solvent particle (at its current
// position, under the grid shift of the collision keyed by *d_step) and every
// site (its cell from the PRE coupling) is counted into its cell; an
// exclusive scan of the counts gives each cell's first slot; a scatter
// places the members; each cell's segment is then put in the canonical order
// (solvent before sites, each by ascending id), so that the result does not
// depend on the order of the atomics.  Keys: a solvent particle is its host
// row (row_begin + tag), a site is ORDER_SITE + its global index.
constexpr unsigned long long ORDER_SITE = 1ull << 62;

template <typename Real>
__device__ __forceinline__ int64_t order_solvent_cell(const DevReplica &r, const int32_t (&S)[3], Real x, Real y,
                                                      Real z)
{
    return (int64_t)r.cell_base + cell_axis(x, S[0], r.L[0]) +
           (int64_t)r.L[0] * (cell_axis(y, S[1], r.L[1]) + r.L[1] * cell_axis(z, S[2], r.L[2]));
}

// SCATTER = false: counts[c] += 1 per member; true: keys[ex[c] + slot] = key
template <typename Real, bool SCATTER>
__global__ void __launch_bounds__(256) k_order_solvent(StepArgs a, int32_t *counts, const int32_t *ex,
                                                       int32_t *cursor, unsigned long long *keys)
{
    const Real *X = (const Real *)a.x, *Y = (const Real *)a.y, *Z = (const Real *)a.z;
    const int64_t step = *a.d_step;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        int32_t S[3];
        grid_shift(r, step, S);
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            const int64_t c = order_solvent_cell(r, S, X[i], Y[i], Z[i]);
            if (!SCATTER) {
                atomicAdd(counts + c, 1);
            } else {
                const int64_t pos = (int64_t)ex[c] + atomicAdd(cursor + c, 1);
                keys[pos] = (unsigned long long)(r.row_begin + a.tag[i]);
            }
        }
    }
}

// sites: one CTA per body
template <bool SCATTER>
__global__ void __launch_bounds__(128) k_order_sites(StepArgs a, int32_t *counts, const int32_t *ex,
                                                     int32_t *cursor, unsigned long long *keys)
{
    const DevBody &B = a.bodies[blockIdx.x];
    const DevReplica r = a.reps[B.rep];
    const int n = a.shapes[B.shape].n_sites;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t g = B.site_begin + j;
        const int64_t c = (int64_t)r.cell_base + a.site_cell[g];
        if (!SCATTER) {
            atomicAdd(counts + c, 1);
        } else {
            const int64_t pos = (int64_t)ex[c] + atomicAdd(cursor + c, 1);
            keys[pos] = ORDER_SITE | (unsigned long long)g;
        }
    }
}

// per cell: insertion sort of its segment by key (segments hold ~10-40),
// then the final ids (solvent: host row; site: n_solvent + site index) and
// the int64 cell starts
__global__ void __launch_bounds__(256) k_order_cells(int64_t n_cells, const int32_t *ex,
                                                     unsigned long long *keys, int64_t n_solvent,
                                                     int64_t *order, int64_t *start)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = ex[c], e = ex[c + 1];
        for (int64_t i = b + 1; i < e; ++i) {
            const unsigned long long k = keys[i];
            int64_t j = i - 1;
            while (j >= b && keys[j] > k) {
                keys[j + 1] = keys[j];
                --j;
            }
            keys[j + 1] = k;
        }
        for (int64_t i = b; i < e; ++i) {
            const unsigned long long k = keys[i];
            order[i] = (k & ORDER_SITE) ? n_solvent + (int64_t)(k & ~ORDER_SITE) : (int64_t)k;
        }
        start[c] = b;
        if (c == n_cells - 1) start[n_cells] = e;
    }
}

void launch_cell_order(const StepArgs &a, int64_t n_solvent, int32_t *counts, int32_t *ex, int32_t *cursor,
                       int32_t *scan_bs, unsigned long long *keys, int64_t *order, int64_t *start, int num_sms,
                       cudaStream_t s)
{
    const int64_t C = a.n_cells;
    cudaMemsetAsync(counts, 0, (C + 1) * sizeof(int32_t), s);
    cudaMemsetAsync(cursor, 0, C * sizeof(int32_t), s);
    const int grid = std::max(1, std::min(a.n_tiles, num_sms * 8));
    if (a.n_tiles > 0) {
        if (a.precision == 1) k_order_solvent<float, false><<<grid, 256, 0, s>>>(a, counts, ex, cursor, keys);
        else k_order_solvent<double, false><<<grid, 256, 0, s>>>(a, counts, ex, cursor, keys);
    }
    if (a.n_bodies > 0) k_order_sites<false><<<a.n_bodies, 128, 0, s>>>(a, counts, ex, cursor, keys);
    launch_scan(counts, ex, C + 1, scan_bs, s);   // counts[C] = 0: ex[C] = number of members
    if (a.n_tiles > 0) {
        if (a.precision == 1) k_order_solvent<float, true><<<grid, 256, 0, s>>>(a, counts, ex, cursor, keys);
        else k_order_solvent<double, true><<<grid, 256, 0, s>>>(a, counts, ex, cursor, keys);
    }
    if (a.n_bodies > 0) k_order_sites<true><<<a.n_bodies, 128, 0, s>>>(a, counts, ex, cursor, keys);
    const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, (int64_t)num_sms * 16));
    k_order_cells<<<cgrid, 256, 0, s>>>(C, ex, keys, n_solvent, order, start);
}

}  // namespace mpcd
