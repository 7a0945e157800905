// Host-state ingest and egress through a stable LSD radix sort.
//
// mpcd_set_state receives the solvent in tag order (spatially random) and
// stores it cell-sorted; mpcd_get_state returns it in tag order again.  Both
// are permutations of up to ~1e8 records.  Scattering every record to its
// destination costs one partially written sector per 4-byte store; instead
// the (key, slot) pairs are sorted by a stable 8-bit-digit radix sort whose
// scatter goes through a shared-memory staging tile (runs of equal digits
// leave the CTA as contiguous stores), and the records are then moved once by
// a gather whose stores are coalesced.  Stability gives the canonical order:
// within a cell, ascending tag.
#include <algorithm>

#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

constexpr int RS_THREADS = 256, RS_ITEMS = 16, RS_TILE = RS_THREADS * RS_ITEMS, RS_BINS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr uint32_t NO_VAL = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    return (1u << (threadIdx.x & 31)) - 1u;
}

// an index outside its array: set ERR_INDEX, note which check fired in the
// second error word (first one wins) and skip the access
__device__ __forceinline__ void bad_index(int *err, int where)
{
    atomicOr(err, ERR_INDEX);
    atomicCAS(err + 1, 0, where);
}

// per-tile digit histogram, stored digit-major: hist[d * n_tiles + tile];
// each thread counts 16 consecutive keys read as four 16-byte vectors
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *keys, int64_t n, int shift,
                                                         int32_t *hist, int n_tiles)
{
    __shared__ int32_t h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
    uint32_t k[RS_ITEMS];
    if (i0 + RS_ITEMS <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(keys + i0);
#pragma unroll
        for (int q = 0; q < RS_ITEMS / 4; ++q) {
            const uint4 w = p[q];
            k[4 * q] = w.x; k[4 * q + 1] = w.y; k[4 * q + 2] = w.z; k[4 * q + 3] = w.w;
        }
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) atomicAdd(&h[(k[j] >> shift) & 255u], 1);
    } else {
        for (int64_t i = i0; i < n; ++i) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one digit pass; offs = exclusive scan of hist.  Warp w
// owns the tile's elements [512 w, 512 w + 512) and ranks them in order with
// warp-private digit counters (match_any per round, warp-level sync only);
// one CTA-wide prefix over the warps then gives tile positions, the tile is
// reordered in shared memory and leaves as runs of contiguous stores.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *keys, const uint32_t *vals,
                                                            uint32_t *okeys, uint32_t *ovals, int64_t n,
                                                            int shift, const int32_t *offs, int n_tiles, int *err)
{
    constexpr int CHUNK = RS_TILE / RS_WARPS;   // elements per warp
    __shared__ int32_t cnt[RS_WARPS][RS_BINS];
    __shared__ uint32_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ int32_t dbase[RS_BINS];
    __shared__ int32_t gbase[RS_BINS];
    __shared__ int32_t wsum[RS_WARPS];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const int nvalid = (int)min((int64_t)RS_TILE, n - base);
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) cnt[w][t] = 0;
    gbase[t] = offs[(int64_t)t * n_tiles + blockIdx.x];
    uint32_t k[RS_ITEMS], v[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + warp * CHUNK + r * 32 + lane;
        k[r] = i < n ? keys[i] : 0xFFFFFFFFu;   // past the end: last digit, last in order
        v[r] = i < n ? vals[i] : NO_VAL;
    }
    __syncthreads();
    int rank[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const uint32_t d = (k[r] >> shift) & 255u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lr = __popc(peers & lanemask_lt());
        const int before = cnt[warp][d];
        __syncwarp();
        if (lr == 0) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + lr;
    }
    __syncthreads();
    // column d: per-warp counts -> offsets within the digit; total per digit
    int tot = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        const int c = cnt[w][t];
        cnt[w][t] = tot;
        tot += c;
    }
    // tile-local exclusive offsets of the digits (block scan of tot)
    {
        int x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        dbase[t] = before + x - tot;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + warp * CHUNK + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (k[r] >> shift) & 255u;
            const int p = dbase[d] + cnt[warp][d] + rank[r];
            if (p < 0 || p >= nvalid) { bad_index(err, 1); continue; }
            sk[p] = k[r];
            sv[p] = v[r];
        }
    }
    __syncthreads();
    for (int j = t; j < nvalid; j += RS_THREADS) {
        const uint32_t key = sk[j];
        const uint32_t d = (key >> shift) & 255u;
        const int64_t pos = (int64_t)gbase[d] + (j - dbase[d]);
        if (pos < 0 || pos >= n) { bad_index(err, 2); continue; }
        okeys[pos] = key;
        ovals[pos] = sv[j];
    }
}

template <typename Real>
__device__ __forceinline__ int floor_cell(Real x, int L)
{
    int c = (int)x;   // x in [0, L): truncation is the floor
    return c < 0 ? 0 : (c >= L ? L - 1 : c);
}

// set_state keys: global cell (no shift) of every real slot's particle, read
// from the host-layout rows; value = host row.  Flags positions outside [0, L).
template <typename Real>
__global__ void k_keys_in(StepArgs a, const Real *xa, uint32_t *keys, uint32_t *vals)
{
    int bad = 0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            const int64_t row = r.row_begin + (i - r.solv_begin);
            const Real x = xa[3 * row], y = xa[3 * row + 1], z = xa[3 * row + 2];
            bad |= !(x >= Real(0) && x < (Real)r.L[0]) || !(y >= Real(0) && y < (Real)r.L[1]) ||
                   !(z >= Real(0) && z < (Real)r.L[2]);
            keys[i] = (uint32_t)(r.cell_base + floor_cell(x, r.L[0]) +
                                 r.L[0] * (floor_cell(y, r.L[1]) + r.L[1] * floor_cell(z, r.L[2])));
            vals[i] = (uint32_t)row;
        }
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// padding slots (after each replica's particles, and the trailing ones):
// key = a value that sorts them to the end of their replica's slot range
__global__ void k_keys_pad(StepArgs a, uint32_t *keys, uint32_t *vals, int64_t nslots, int mode,
                           uint32_t out_key)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n_rep; r += gridDim.x * blockDim.x) {
        const DevReplica R = a.reps[r];
        const int64_t b = R.solv_begin + R.n_solvent;
        const int64_t e = r + 1 < a.n_rep ? a.reps[r + 1].solv_begin : nslots;
        const uint32_t key = mode == 0 ? (uint32_t)(R.cell_base + R.L[0] * R.L[1] * R.L[2] - 1) : out_key;
        for (int64_t i = b; i < e; ++i) {
            keys[i] = key;
            vals[i] = NO_VAL;
        }
    }
}

// 8-word record load / store as 16-byte vectors
__device__ __forceinline__ void rec_load(const float *r, float (&o)[6])
{
    const float4 a = reinterpret_cast<const float4 *>(r)[0], b = reinterpret_cast<const float4 *>(r)[1];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
}
__device__ __forceinline__ void rec_load(const double *r, double (&o)[6])
{
    const double2 *p = reinterpret_cast<const double2 *>(r);
    const double2 a = p[0], b = p[1], c = p[2];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y;
}
__device__ __forceinline__ void rec_store(float *r, const float (&o)[6])
{
    reinterpret_cast<float4 *>(r)[0] = make_float4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<float4 *>(r)[1] = make_float4(o[4], o[5], 0.0f, 0.0f);
}
__device__ __forceinline__ void rec_store(double *r, const double (&o)[6])
{
    double2 *p = reinterpret_cast<double2 *>(r);
    p[0] = make_double2(o[0], o[1]);
    p[1] = make_double2(o[2], o[3]);
    p[2] = make_double2(o[4], o[5]);
    p[3] = make_double2(0.0, 0.0);
}

// host rows -> 8-word records {x, y, z, vx, vy, vz, 0, 0} (coalesced), so
// that the permuting gather reads one aligned 32-byte (P32) or 64-byte (P64)
// record per particle instead of six scattered words
template <typename Real>
__global__ void k_pack_rows(const Real *xa, const Real *va, Real *rec, int64_t n_rows)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_rows; j += stride) {
        Real o[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) { o[k] = xa[3 * j + k]; o[3 + k] = va[3 * j + k]; }
        rec_store(rec + 8 * j, o);
    }
}

// set_state gather: sorted position i holds the host row of the record that
// belongs in slot i; padding slots get zeros and the padding tag
template <typename Real>
__global__ void k_gather_in(StepArgs a, const Real *rec, const uint32_t *vals, int64_t nslots, int64_t n_rows)
{
    Real *X[3] = {(Real *)a.x, (Real *)a.y, (Real *)a.z};
    Real *V[3] = {(Real *)a.vx, (Real *)a.vy, (Real *)a.vz};
    // four records in flight per thread: all loads are issued before any store
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nslots; i0 += 4 * stride) {
        Real r[4][6];
        uint32_t row[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * stride;
            row[u] = i < nslots ? vals[i] : NO_VAL;
            if (row[u] != NO_VAL && (int64_t)row[u] >= n_rows) {
                bad_index(a.d_err, 3);
                row[u] = NO_VAL - 1;   // skip: neither a record nor padding
            }
            if ((int64_t)row[u] < n_rows) rec_load(rec + 8 * (int64_t)row[u], r[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= nslots || row[u] == NO_VAL - 1) continue;
            if (row[u] == NO_VAL) {
#pragma unroll
                for (int k = 0; k < 3; ++k) { X[k][i] = Real(0); V[k][i] = Real(0); }
                a.tag[i] = PAD_TAG;
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) { X[k][i] = r[u][k]; V[k][i] = r[u][3 + k]; }
            }
        }
    }
}

// the tag of every real slot: host row - the replica's first row
__global__ void k_tags_in(StepArgs a, const uint32_t *vals)
{
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            const int64_t tag = (int64_t)vals[i] - r.row_begin;
            if (tag < 0 || tag >= r.n_solvent) { bad_index(a.d_err, 4); continue; }
            a.tag[i] = (uint32_t)tag;
        }
    }
}

// get_state keys: host row of every real slot (padding gets out_key = N_s)
__global__ void k_keys_out(StepArgs a, uint32_t *keys, uint32_t *vals)
{
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const DevReplica r = a.reps[tl.rep];
        for (int64_t i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            keys[i] = (uint32_t)(r.row_begin + a.tag[i]);
            vals[i] = (uint32_t)i;
        }
    }
}

// storage slots -> 8-word records (coalesced), for the egress gather
template <typename Real>
__global__ void k_pack_slots(StepArgs a, Real *rec, int64_t nslots)
{
    const Real *X[3] = {(const Real *)a.x, (const Real *)a.y, (const Real *)a.z};
    const Real *V[3] = {(const Real *)a.vx, (const Real *)a.vy, (const Real *)a.vz};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nslots; p += stride) {
        Real o[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) { o[k] = X[k][p]; o[3 + k] = V[k][p]; }
        rec_store(rec + 8 * p, o);
    }
}

// get_state gather: host row i from the record of slot vals[i], stored row by row
template <typename Real>
__global__ void k_gather_out(const uint32_t *vals, const Real *rec, Real *xa, Real *va, int64_t row0,
                             int64_t n_rows, int64_t nslots, int *err)
{
    // rows [row0, n_rows); four records in flight per thread: all loads are
    // issued before any store
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n_rows; i0 += 4 * stride) {
        Real r[4][6];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * stride;
            const int64_t p = i < n_rows ? (int64_t)vals[i] : -1;
            ok[u] = p >= 0 && p < nslots;
            if (p >= nslots) bad_index(err, 5);
            if (ok[u]) rec_load(rec + 8 * p, r[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * stride;
            if (!ok[u]) continue;
#pragma unroll
            for (int k = 0; k < 3; ++k) { xa[3 * i + k] = r[u][k]; va[3 * i + k] = r[u][3 + k]; }
        }
    }
}

int grid_for(int64_t n, int per_block, int cap)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, cap));
}

}  // namespace

size_t radix_hist_ints(int64_t n)
{
    return (size_t)RS_BINS * (size_t)std::max<int64_t>(1, (n + RS_TILE - 1) / RS_TILE);
}

int key_bits(uint64_t max_key)
{
    int b = 1;
    while (b < 32 && (max_key >> b) != 0) ++b;
    return b;
}

int launch_radix_sort(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, int64_t n, int nbits,
                      int32_t *hist, int32_t *hist_ex, int32_t *scan_bs, int *err, cudaStream_t s)
{
    if (n <= 0) return 0;
    const int n_tiles = (int)((n + RS_TILE - 1) / RS_TILE);
    int in_b = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        const uint32_t *ki = in_b ? kB : kA, *vi = in_b ? vB : vA;
        uint32_t *ko = in_b ? kA : kB, *vo = in_b ? vA : vB;
        k_rs_hist<<<n_tiles, RS_THREADS, 0, s>>>(ki, n, shift, hist, n_tiles);
        launch_scan(hist, hist_ex, (int64_t)RS_BINS * n_tiles, scan_bs, s);
        k_rs_scatter<<<n_tiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, hist_ex, n_tiles, err);
        in_b ^= 1;
    }
    return in_b;
}

void launch_keys_in(const StepArgs &a, const void *xa, uint32_t *keys, uint32_t *vals, int64_t nslots,
                    cudaStream_t s)
{
    k_keys_pad<<<grid_for(a.n_rep, 128, 1024), 128, 0, s>>>(a, keys, vals, nslots, 0, 0u);
    if (a.n_tiles == 0) return;
    if (a.precision == 1) k_keys_in<float><<<a.n_tiles, 256, 0, s>>>(a, (const float *)xa, keys, vals);
    else k_keys_in<double><<<a.n_tiles, 256, 0, s>>>(a, (const double *)xa, keys, vals);
}

void launch_pack_rows(const StepArgs &a, const void *xa, const void *va, void *rec, int64_t n_rows, int num_sms,
                      cudaStream_t s)
{
    if (n_rows == 0) return;
    const int grid = grid_for(n_rows, 256, num_sms * 8);
    if (a.precision == 1) k_pack_rows<float><<<grid, 256, 0, s>>>((const float *)xa, (const float *)va, (float *)rec, n_rows);
    else k_pack_rows<double><<<grid, 256, 0, s>>>((const double *)xa, (const double *)va, (double *)rec, n_rows);
}

void launch_gather_in(const StepArgs &a, const void *rec, const uint32_t *vals, int64_t nslots, int64_t n_rows,
                      int num_sms, cudaStream_t s)
{
    const int grid = grid_for(nslots, 256, num_sms * 8);
    if (a.precision == 1) k_gather_in<float><<<grid, 256, 0, s>>>(a, (const float *)rec, vals, nslots, n_rows);
    else k_gather_in<double><<<grid, 256, 0, s>>>(a, (const double *)rec, vals, nslots, n_rows);
    if (a.n_tiles) k_tags_in<<<a.n_tiles, 256, 0, s>>>(a, vals);
}

void launch_keys_out(const StepArgs &a, uint32_t *keys, uint32_t *vals, int64_t nslots, uint32_t n_rows,
                     cudaStream_t s)
{
    k_keys_pad<<<grid_for(a.n_rep, 128, 1024), 128, 0, s>>>(a, keys, vals, nslots, 1, n_rows);
    if (a.n_tiles) k_keys_out<<<a.n_tiles, 256, 0, s>>>(a, keys, vals);
}

void launch_pack_slots(const StepArgs &a, void *rec, int64_t nslots, int num_sms, cudaStream_t s)
{
    const int gp = grid_for(nslots, 256, num_sms * 8);
    if (a.precision == 1) k_pack_slots<float><<<gp, 256, 0, s>>>(a, (float *)rec, nslots);
    else k_pack_slots<double><<<gp, 256, 0, s>>>(a, (double *)rec, nslots);
}

void launch_gather_rows(const StepArgs &a, const uint32_t *vals, const void *rec, void *xa, void *va, int64_t row0,
                        int64_t row1, int64_t nslots, int num_sms, cudaStream_t s)
{
    if (row1 <= row0) return;
    const int grid = grid_for(row1 - row0, 256, num_sms * 8);
    if (a.precision == 1)
        k_gather_out<float><<<grid, 256, 0, s>>>(vals, (const float *)rec, (float *)xa, (float *)va, row0, row1,
                                                 nslots, a.d_err);
    else
        k_gather_out<double><<<grid, 256, 0, s>>>(vals, (const double *)rec, (double *)xa, (double *)va, row0, row1,
                                                  nslots, a.d_err);
}

}  // namespace mpcd
