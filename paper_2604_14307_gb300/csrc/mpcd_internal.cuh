// Internal definitions of the sm_103a MPCD library (not part of the C ABI).
//
// Data layout in HBM
//   solvent   SoA x, y, z, vx, vy, vz (float for P32, double for P64) plus a
//             uint32 tag, double-buffered for the periodic spatial re-sort.
//             Each replica owns slots [solv_begin, solv_begin + n_solvent),
//             solv_begin a multiple of 8; padding slots carry tag 0xFFFFFFFF.
//   cells     `sums`:   NW word arrays of n_cells entries (int64 fixed point
//                       for P32, double for P64), zero between collisions;
//             `params`: one record per cell (32 B for P32, 64 B for P64):
//                       u, kappa (< 0 marks a cell that does not collide),
//                       and the SRD axis or the AT mean noise.
//   bodies    one FP64 record per body (R, q, P, L, F, T).
//   sites     thermalised velocity (3 x Real SoA) and cell of every site,
//             written by the PRE coupling and read by the POST coupling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpcd {

// Counter word 2 of every random draw (stream tags).
enum : uint32_t { TAG_SHIFT = 1, TAG_AXIS = 2, TAG_THERMO = 3, TAG_THERMO_ODD = 4,
                  TAG_SITE = 5, TAG_AT = 6 };
// Bits of the device error word.
enum : int { ERR_POSITION = 1, ERR_CELL = 2 };

constexpr uint32_t PAD_TAG = 0xFFFFFFFFu;

struct DevReplica {
    int32_t L[3];
    int32_t cell_base;      // first global cell of the replica
    int64_t solv_begin;     // first storage slot
    int64_t n_solvent;
    int64_t body_begin, body_end;
    int64_t site_begin;     // first global site index
    int64_t row_begin;      // first row of the replica in host (tag-ordered) arrays
    uint32_t key0, key1;    // Philox key: (seed_lo, seed_hi ^ replica)
};

struct Tile {               // a contiguous work range inside one replica
    int32_t rep;
    int32_t pad;
    int64_t begin, end;
};

struct DevShape {
    int64_t site_begin;     // into the template tables
    int64_t cent_begin;
    int32_t n_sites, n_cent;
    double M;               // total site mass
    double Ihat[3];         // principal moments of the sites
    double wca_d;           // centre diameter
    double bound;           // largest centre distance from the COM
};

struct DevBody {
    double R[3];
    double q[4];
    double P[3];            // linear momentum (Eq. 3)
    double Lm[3];           // space-frame angular momentum (Eq. 4)
    double F[3];
    double T[3];
    int32_t shape, rep;
    int64_t site_begin;     // global index of the body's first site
};

// Arguments shared by every kernel of a step (passed by value).
struct StepArgs {
    int32_t precision, rule, thermostat, naive;
    double kT, dt, m_solvent, cos_a, sin_a;
    float kTf, dtf, m_solvent_f, cos_af, sin_af;
    long long w0_solvent;           // fixed-point count|mass word of a solvent particle
    const DevReplica *reps;
    int32_t n_rep;
    const Tile *tiles;              // solvent tiles
    int32_t n_tiles;
    const Tile *ctiles;             // cell tiles
    int32_t n_ctiles;
    void *x, *y, *z, *vx, *vy, *vz; // current solvent buffers
    uint32_t *tag;
    void *sums;                     // [nw][n_cells]
    void *params;                   // [n_cells] records
    void *dbg_sums;                 // copy of the sums when debugging, else null
    int64_t n_cells;
    int32_t nw;
    DevBody *bodies;
    float4 *bpos;                   // per body: R in float, bounding radius (force prefilter)
    int32_t n_bodies;
    const DevShape *shapes;
    const double *tb;               // template offsets [sites][3]
    const float *tbf;               // the same rounded to float
    const double *tm;               // template masses
    const float *tmf;
    const double *tcent;            // WCA centres [centres][3]
    double max_wca_d;               // largest centre diameter of any shape
    void *site_v;                   // [3][n_sites] SoA
    int32_t *site_cell;             // replica-local cell of each site
    int64_t n_sites;
    const int64_t *d_step;          // completed steps (device)
    int *d_err;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), GPU/host implementation.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
#else
        uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += W0;
        k1 += W1;
    }
    return c;
}

__host__ __device__ __forceinline__ uint4 draw(const DevReplica &r, int64_t step, uint32_t id,
                                               uint32_t tag, uint32_t j)
{
    return philox4x32_10(make_uint4((uint32_t)step, id, tag, j), r.key0, r.key1);
}

// Integer grid shift S in [-2^19, 2^19) per axis; s = S 2^-20 (Sec. II.A).
__host__ __device__ __forceinline__ void grid_shift(const DevReplica &r, int64_t step, int32_t S[3])
{
    uint4 w = draw(r, step, 0u, TAG_SHIFT, 0u);
    S[0] = (int32_t)(w.x >> 12) - (1 << 19);
    S[1] = (int32_t)(w.y >> 12) - (1 << 19);
    S[2] = (int32_t)(w.z >> 12) - (1 << 19);
}

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the kernel translation units).
// ---------------------------------------------------------------------------
enum : int { SOLV_COLLIDE = 1, SOLV_STREAM = 2, SOLV_BIN = 4 };

struct LaunchCfg {
    int block;      // threads per CTA of the solvent pass
    int grid;       // CTAs (persistent over tiles)
};

// solvent pass (kernels_solvent.cu)
void launch_solvent(const StepArgs &a, int flags, LaunchCfg cfg, cudaStream_t s);
void launch_params(const StepArgs &a, int grid, cudaStream_t s);
void launch_aos_to_soa(const StepArgs &a, const void *xaos, const void *vaos, cudaStream_t s);
void launch_soa_to_aos(const StepArgs &a, void *xaos, void *vaos, const int64_t *out_off,
                       cudaStream_t s);
void launch_solvent_diag(const StepArgs &a, double *acc, cudaStream_t s);
// re-sort (kernels_solvent.cu)
void launch_sort_count(const StepArgs &a, int32_t *counts, cudaStream_t s);
void launch_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *block_sums, cudaStream_t s);
void launch_sort_scatter(const StepArgs &a, const int32_t *offsets, int32_t *cursor,
                         void *const dst[6], uint32_t *dst_tag, cudaStream_t s);
void launch_sort_canonical(const StepArgs &a, void *const arr[6], uint32_t *tag,
                           const int32_t *offsets, cudaStream_t s);
size_t scan_block_sums_size(int64_t n);

// bodies and sites (kernels_bodies.cu)
void launch_body_md(const StepArgs &a, cudaStream_t s);
void launch_body_force(const StepArgs &a, int kick, cudaStream_t s);
void launch_sites_pre(const StepArgs &a, int max_sites, cudaStream_t s);
void launch_sites_post(const StepArgs &a, int max_sites, cudaStream_t s);
void launch_advance_step(const StepArgs &a, cudaStream_t s);
void launch_body_diag(const StepArgs &a, double *acc, cudaStream_t s);
cudaError_t configure_body_kernels(int max_sites, int precision);

}  // namespace mpcd
