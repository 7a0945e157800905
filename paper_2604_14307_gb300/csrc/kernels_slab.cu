// Kernels of the spatial domain decomposition of one box into slabs along z
// (one context per slab): the split of a context's solvent into the particles
// that stay in its slab and those that left it (order-preserving stream
// compaction per fixed 2048-particle tile), the upload of arriving particles,
// the export of the leavers, the addition of a neighbour's partial cell words,
// and the per-body momentum transfer summed over the slab's own sites.
#include <algorithm>

#include "mpcd_internal.cuh"

namespace mpcd {

constexpr int SLAB_THREADS = 256;

template <typename Real>
__device__ __forceinline__ bool slab_leaves(Real z, int zlo, int zhi)
{
    return !(z >= (Real)zlo && z < (Real)zhi);
}

// leavers per io tile (z outside [zlo, zhi))
template <typename Real>
__global__ void __launch_bounds__(SLAB_THREADS) k_slab_count(StepArgs a, int zlo, int zhi, int32_t *leave)
{
    __shared__ int wsum[SLAB_THREADS / 32];
    const Tile tl = a.tiles[blockIdx.x];
    const Real *Z = (const Real *)a.z;
    int n = 0;
    for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += SLAB_THREADS) n += slab_leaves(Z[i], zlo, zhi);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SLAB_THREADS / 32; ++w) t += wsum[w];
        leave[blockIdx.x] = t;
    }
}

// order-preserving split of each tile: kept particles to dst[] at the tile's
// kept offset, leavers to exp[] at its leaver offset (leave_ex: exclusive scan
// of the per-tile leaver counts over the tiles)
template <typename Real>
__global__ void __launch_bounds__(SLAB_THREADS) k_slab_split(StepArgs a, int zlo, int zhi, const int32_t *leave_ex,
                                                              Real *d0, Real *d1, Real *d2, Real *d3, Real *d4,
                                                              Real *d5, uint32_t *dtag, Real *e0, Real *e1, Real *e2,
                                                              Real *e3, Real *e4, Real *e5, uint32_t *etag)
{
    __shared__ int wcnt[SLAB_THREADS / 32];
    const Tile tl = a.tiles[blockIdx.x];
    const DevReplica r = a.reps[tl.rep];
    const Real *S[6] = {(const Real *)a.x, (const Real *)a.y, (const Real *)a.z,
                        (const Real *)a.vx, (const Real *)a.vy, (const Real *)a.vz};
    Real *D[6] = {d0, d1, d2, d3, d4, d5};
    Real *E[6] = {e0, e1, e2, e3, e4, e5};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t keep_at = (tl.begin - r.solv_begin) - leave_ex[blockIdx.x] + r.solv_begin;
    int64_t leave_at = leave_ex[blockIdx.x];
    for (int64_t base = tl.begin; base < tl.end; base += SLAB_THREADS) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < tl.end;
        const bool out = valid && slab_leaves(S[2][i], zlo, zhi);
        const unsigned bo = __ballot_sync(0xffffffffu, out), bv = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) wcnt[warp] = __popc(bo);
        __syncthreads();
        int before_out = 0, total_out = 0;
        for (int w = 0; w < SLAB_THREADS / 32; ++w) {
            if (w < warp) before_out += wcnt[w];
            total_out += wcnt[w];
        }
        const unsigned lt = (1u << lane) - 1u;
        const int rank_out = before_out + __popc(bo & lt);
        const int idx = (int)(i - base);
        const int rank_in = idx - rank_out;
        if (valid) {
            if (out) {
                const int64_t o = leave_at + rank_out;
                for (int k = 0; k < 6; ++k) E[k][o] = S[k][i];
                etag[o] = a.tag[i];
            } else {
                const int64_t o = keep_at + rank_in;
                for (int k = 0; k < 6; ++k) D[k][o] = S[k][i];
                dtag[o] = a.tag[i];
            }
        }
        const int nvalid = (int)min((int64_t)SLAB_THREADS, tl.end - base);
        (void)bv;
        keep_at += nvalid - total_out;
        leave_at += total_out;
        __syncthreads();
    }
}

// rows of host-layout arrays (x[n][3], v[n][3], tags[n]) into storage slots
// [at, at + n) of the current buffers
template <typename Real>
__global__ void k_slab_put(StepArgs a, const Real *xa, const Real *va, const uint32_t *tags, int64_t n, int64_t at)
{
    Real *X[6] = {(Real *)a.x, (Real *)a.y, (Real *)a.z, (Real *)a.vx, (Real *)a.vy, (Real *)a.vz};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            X[k][at + i] = xa[3 * i + k];
            X[3 + k][at + i] = va[3 * i + k];
        }
        a.tag[at + i] = tags[i];
    }
}

// SoA rows [0, n) of e[6], etag -> host layout x[n][3], v[n][3], tags[n]
template <typename Real>
__global__ void k_slab_pack(const Real *e0, const Real *e1, const Real *e2, const Real *e3, const Real *e4,
                            const Real *e5, const uint32_t *etag, int64_t n, Real *xa, Real *va, uint32_t *tags)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        xa[3 * i] = e0[i]; xa[3 * i + 1] = e1[i]; xa[3 * i + 2] = e2[i];
        va[3 * i] = e3[i]; va[3 * i + 1] = e4[i]; va[3 * i + 2] = e5[i];
        tags[i] = etag[i];
    }
}

// sums[k][cell0 + i] += add[k][i] for the nw word arrays (integer words: exact)
template <typename W>
__global__ void k_words_add(W *sums, int nw, int64_t C, int64_t cell0, int64_t ncell, const W *add)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < nw; ++k) sums[k * C + cell0 + i] += add[k * ncell + i];
}

// per-body transfer of this context's own sites, [n_bodies][6] in FP64
template <typename Real>
__global__ void k_body_partial(StepArgs a, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const Real *in = reinterpret_cast<const Real *>(a.partial) + (int64_t)i * SITE_WARPS * 6;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < SITE_WARPS; ++w)
        for (int k = 0; k < 6; ++k) s[k] += (double)in[w * 6 + k];
    for (int k = 0; k < 6; ++k) out[6 * i + k] = s[k];
}

__global__ void k_body_apply(StepArgs a, const double *dpl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    DevBody *o = a.bodies + i;
    for (int k = 0; k < 3; ++k) {
        o->P[k] += dpl[6 * i + k];
        o->Lm[k] += dpl[6 * i + 3 + k];
    }
}

void launch_slab_count(const StepArgs &a, int zlo, int zhi, int32_t *leave, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    if (a.precision == 1) k_slab_count<float><<<a.n_tiles, SLAB_THREADS, 0, s>>>(a, zlo, zhi, leave);
    else k_slab_count<double><<<a.n_tiles, SLAB_THREADS, 0, s>>>(a, zlo, zhi, leave);
}

void launch_slab_split(const StepArgs &a, int zlo, int zhi, const int32_t *leave_ex, void *const dst[6],
                       uint32_t *dst_tag, void *const exp[6], uint32_t *exp_tag, cudaStream_t s)
{
    if (a.n_tiles == 0) return;
    if (a.precision == 1)
        k_slab_split<float><<<a.n_tiles, SLAB_THREADS, 0, s>>>(
            a, zlo, zhi, leave_ex, (float *)dst[0], (float *)dst[1], (float *)dst[2], (float *)dst[3],
            (float *)dst[4], (float *)dst[5], dst_tag, (float *)exp[0], (float *)exp[1], (float *)exp[2],
            (float *)exp[3], (float *)exp[4], (float *)exp[5], exp_tag);
    else
        k_slab_split<double><<<a.n_tiles, SLAB_THREADS, 0, s>>>(
            a, zlo, zhi, leave_ex, (double *)dst[0], (double *)dst[1], (double *)dst[2], (double *)dst[3],
            (double *)dst[4], (double *)dst[5], dst_tag, (double *)exp[0], (double *)exp[1], (double *)exp[2],
            (double *)exp[3], (double *)exp[4], (double *)exp[5], exp_tag);
}

void launch_slab_put(const StepArgs &a, const void *xa, const void *va, const uint32_t *tags, int64_t n, int64_t at,
                     int num_sms, cudaStream_t s)
{
    if (n <= 0) return;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
    if (a.precision == 1) k_slab_put<float><<<grid, 256, 0, s>>>(a, (const float *)xa, (const float *)va, tags, n, at);
    else k_slab_put<double><<<grid, 256, 0, s>>>(a, (const double *)xa, (const double *)va, tags, n, at);
}

void launch_slab_pack(int precision, void *const exp[6], const uint32_t *exp_tag, int64_t n, void *xa, void *va,
                      uint32_t *tags, int num_sms, cudaStream_t s)
{
    if (n <= 0) return;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
    if (precision == 1)
        k_slab_pack<float><<<grid, 256, 0, s>>>((const float *)exp[0], (const float *)exp[1], (const float *)exp[2],
                                               (const float *)exp[3], (const float *)exp[4], (const float *)exp[5],
                                               exp_tag, n, (float *)xa, (float *)va, tags);
    else
        k_slab_pack<double><<<grid, 256, 0, s>>>((const double *)exp[0], (const double *)exp[1],
                                                (const double *)exp[2], (const double *)exp[3],
                                                (const double *)exp[4], (const double *)exp[5], exp_tag, n,
                                                (double *)xa, (double *)va, tags);
}

void launch_words_add(int precision, void *sums, int nw, int64_t C, int64_t cell0, int64_t ncell, const void *add,
                      int num_sms, cudaStream_t s)
{
    if (ncell <= 0) return;
    const int grid = (int)std::min<int64_t>((ncell + 255) / 256, (int64_t)num_sms * 8);
    if (precision == 1)
        k_words_add<long long><<<grid, 256, 0, s>>>((long long *)sums, nw, C, cell0, ncell, (const long long *)add);
    else
        k_words_add<double><<<grid, 256, 0, s>>>((double *)sums, nw, C, cell0, ncell, (const double *)add);
}

void launch_body_partial(const StepArgs &a, double *out, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    if (a.precision == 1) k_body_partial<float><<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a, out);
    else k_body_partial<double><<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a, out);
}

void launch_body_apply(const StepArgs &a, const double *dpl, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    k_body_apply<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a, dpl);
}

}  // namespace mpcd
