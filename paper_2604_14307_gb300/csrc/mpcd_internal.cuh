// Internal definitions of the sm_103a MPCD library (not part of the C ABI).
//
// Data layout in HBM
//   solvent   SoA x, y, z, vx, vy, vz (float for P32, double for P64) plus a
//             uint32 tag, double-buffered for the periodic spatial re-sort.
//             Each replica owns slots [solv_begin, solv_begin + n_solvent),
//             solv_begin a multiple of 8; padding slots carry tag 0xFFFFFFFF.
//   cells     `sums`:   NW word arrays of n_cells entries (SoA: the lanes of a
//                       warp handle neighbouring cells, so their atomics share
//                       sectors): int64 fixed point for P32 (3 words SRD, 4 AT),
//                       double for P64.  Zero between collisions.
//             `params`: one record per cell (32 B for P32, 64 B for P64):
//                       u, kappa (< 0 marks a cell that does not collide),
//                       and the SRD axis or the AT mean noise.
//   bodies    one FP64 record per body (R, q, P, L, F, T, unwrapped
//             displacement D); the space-frame offsets of every WCA centre
//             (FP64 and float copies), recomputed once per pose.
//   sites     thermalised velocity (3 x Real SoA) and cell of every site,
//             written by the PRE coupling and read by the POST coupling.
//   protocols (allocated on first use) the exchange's key histogram, member
//             lists and candidates; the velocity-profile sums; the per-body
//             autocorrelation rings and sums.
//   +a        (angular-momentum-conserving variants only) ANG_WORDS more words
//             per cell, one AngParams record per cell, one grid shift per
//             replica.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpcd {

// Counter word 2 of every random draw (stream tags).
enum : uint32_t { TAG_SHIFT = 1, TAG_AXIS = 2, TAG_THERMO = 3, TAG_THERMO_ODD = 4,
                  TAG_SITE = 5, TAG_AT = 6, TAG_THERMO_MT = 7 };
// Bits of the device error word.
enum : int { ERR_POSITION = 1, ERR_CELL = 2, ERR_TIMEOUT = 4, ERR_INDEX = 8, ERR_RNEMD = 16 };

constexpr uint32_t PAD_TAG = 0xFFFFFFFFu;
constexpr int NLIST_MAX = 96;       // neighbour-list capacity per body
constexpr float NLIST_SKIN = 0.5f;  // Verlet skin of the body neighbour lists
constexpr int POSE_W = 20;          // words of a pose record
constexpr int SITE_THREADS = 128;   // threads of the per-body site kernels
constexpr int SITE_WARPS = SITE_THREADS / 32;

struct DevReplica {
    int32_t L[3];
    int32_t cell_base;      // first global cell of the replica
    int64_t solv_begin;     // first storage slot
    int64_t n_solvent;
    int64_t body_begin, body_end;
    int64_t site_begin;     // first global site index
    int64_t row_begin;      // first row of the replica in host (tag-ordered) arrays
    int64_t site_id_base;   // id of the replica's first site in its random streams: the
                            // solvent count of the whole box (a slab of a box holds fewer)
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
    double D[3];            // displacement since mpcd_set_state, unwrapped (diffusion)
    int32_t shape, rep;
    int64_t site_begin;     // global index of the body's first site
    int64_t cent_begin;     // global index of the body's first WCA centre (rotated-centre buffers)
};

// Arguments shared by every kernel of a step (passed by value).
struct StepArgs {
    int32_t precision, rule, thermostat, naive;
    double kT, dt, m_solvent, cos_a, sin_a;
    float kTf, dtf, m_solvent_f, cos_af, sin_af;
    long long qm_solvent, qm_site;  // round(m 2^24) of the solvent and of the sites (P32)
    float m_site_f;                 // site mass of the P32 form (uniform)
    double m_site;                  // the same in double (the +a variants need a uniform site mass)
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
    float4 *bpos_build;             // positions when the neighbour lists were built
    int32_t *nlist;                 // [n_bodies][NLIST_MAX] neighbour candidates, ascending
    int32_t *ncount;                // candidates per body, -1 after an overflow
    int *nl_dirty;                  // set when a body moved more than half the skin
    float *pose32;                  // per body [POSE_W]: Q (9), R (3), V (3), omega (3) in float
    double *pose64;                 // the same in double
    void *partial;                  // per body [SITE_WARPS][6] transfer partial sums (Real)
    int32_t n_bodies;
    const DevShape *shapes;
    const double *tb;               // template offsets [sites][3]
    const float *tbf;               // the same rounded to float
    const double *tm;               // template masses
    const float *tmf;
    const double *tcent;            // WCA centres [centres][3]
    double max_wca_d;               // largest centre diameter of any shape
    int32_t max_cent;               // most WCA centres of any shape
    double *cent64;                 // per body centre: Q c in the space frame [n][3] (this step's pose)
    float4 *cent32;                 // the same rounded to float
    void *site_v;                   // [3][n_sites] SoA
    int32_t *site_cell;             // replica-local cell of each site
    int64_t n_sites;
    int32_t accel;                  // constant-force streaming of the solvent (below)
    double ah[3];                   // its half-step velocity change a dt / 2 (P64)
    float ahf[3];                   // the same rounded to float (P32)
    double fext[3];                 // constant force on every body at its centre of mass
    const int64_t *d_step;          // completed steps (device)
    int32_t step_offset;            // added to *d_step by the site PRE pass (1 when it runs
                                    // for the next step before the counter advances)
    int *d_err;
    int *tile_ctr;                  // tile counter of the staged solvent pass (null: round robin)
    // slab of a decomposed box: only the sites with z in [site_zlo, site_zhi)
    // are binned and transfer their momentum here (site_own = 0: every site)
    int32_t site_own, site_zlo, site_zhi;
    // angular-momentum-conserving variants (null when off)
    void *ang_words;                // [ANG_WORDS][n_cells]
    const void *ang_params;         // [n_cells] AngParams records
    int4 *ang_shift;                // [n_rep] grid shift of the current collision
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
// Fixed-point conversions on the integer/FP32 pipes.  On sm_103a the 64-bit
// integer <-> float conversion instructions run at the reduced FP64 rate, so
// they are written out with bit operations here.
// ---------------------------------------------------------------------------
// round-half-even(f * 2^S) as int64, identical to __float2ll_rn(f * 2^S)
// while |f * 2^S| < 2^62 (every physical velocity, energy and mass term)
template <int S>
__device__ __forceinline__ long long qfix(float f)
{
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xFFu);
    const uint32_t man = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = e - 150 + S;             // f * 2^S = man * 2^(e - 150 + S)
    long long q;
    if (e == 0 || sh < -25) {
        q = 0;                              // |f * 2^40| < 1/2 rounds to 0
    } else if (sh >= 0) {
        q = (long long)man << (sh < 38 ? sh : 38);
    } else {
        const int rs = -sh;                 // 1..25
        uint32_t qq = rs < 32 ? man >> rs : 0u;
        const uint32_t rem = man & ((1u << rs) - 1u), half = 1u << (rs - 1);
        qq += (rem > half || (rem == half && (qq & 1u))) ? 1u : 0u;
        q = (long long)qq;
    }
    return (b >> 31) ? -q : q;
}
__device__ __forceinline__ long long q40(float f) { return qfix<40>(f); }
__device__ __forceinline__ long long pack2(long long hi, long long lo)
{
    return (long long)((unsigned long long)hi << 32) + lo;
}

// The P32 cell words (SoA arrays of n_cells int64), exact sums over a cell of
//   w0 = p_x + 2^48 [solvent],  w1 = p_y + 2^48 [site],  w2 = p_z
//                                                  p = round(fl32(m v) 2^32)
//   SRD: w3 = round(e 2^28), e = fl32(fl32(fl32(px vx) + fl32(py vy)) + fl32(pz vz))
//   AT:  w3, w4, w5 = q                            q = round(fl32(m xi) 2^32)
// The low 48 bits of w0 and w1 hold the signed momentum sums, the high 16 bits
// the cell's solvent and site counts.  The 2^-32 quantum is below one float32
// ulp of every |m v| >= 2^-9, so the momentum sums are the exact sums of the
// float32 momenta (a term below 2^-9 is rounded by at most 2^-33).  Limits per
// cell: |sum m v_a| < 2^15, at most 65535 solvent particles and 65535 sites.
template <int RULE> struct Words32 { static constexpr int n = RULE == 0 ? 4 : 6; };
constexpr int MAX_WORDS32 = 6;
constexpr long long COUNT48 = 1LL << 48;

// round-half-even(f 2^20) for |f 2^20| < 2^31: the power-of-two scale is
// exact, so one 32-bit conversion gives the same integer as qfix<20> (the
// momentum terms of the angular-momentum words)
__device__ __forceinline__ long long q20(float f) { return (long long)__float2int_rn(__fmul_rn(f, 1048576.0f)); }

// floor(t) for |t| < 2^22 without a conversion instruction: t + 1.5 2^23
// rounded toward -inf lies in [2^23, 2^24), where the float32 spacing is 1, so
// it is 1.5 2^23 + floor(t) exactly; its low mantissa bits hold floor(t) and
// subtracting 1.5 2^23 again gives floor(t) as a float, exactly (Sterbenz).
constexpr float FLOOR_MAGIC = 12582912.0f;     // 1.5 2^23, bits 0x4B400000
__device__ __forceinline__ float floor_magic(float t) { return __fadd_rd(t, FLOOR_MAGIC); }
__device__ __forceinline__ int floor_magic_int(float m) { return __float_as_int(m) - 0x4B400000; }

// round-half-even(f 2^32) as int64 for |f| < 2^14, with one 32-bit conversion.
// t = f 2^8 is exact; with h = floor(t), f 2^32 = h 2^24 + (t - h) 2^24.
// For |t| >= 1/2 (and t >= 0) the difference r = t - h is exact and r 2^24
// is an integer or is rounded once by the conversion; for t in [-1/2, 0)
// r = t + 1 lies in [1/2, 1), where float32 has the spacing 2^-24, so forming
// r rounds t 2^24 + 2^24 to an integer - the rounding the result needs (ties
// to even: 2^24 is even).  Identical to qfix<32>(f) on that range.
__device__ __forceinline__ long long q32(float f)
{
    const float t = __fmul_rn(f, 256.0f);
    const float hm = floor_magic(t);
    const float r = __fsub_rn(t, __fsub_rn(hm, FLOOR_MAGIC));
    const int h = floor_magic_int(hm);
    const int l = __float2int_rn(__fmul_rn(r, 16777216.0f));
    return (long long)((unsigned long long)(long long)h << 24) + l;
}

// round-half-even(e 2^28) as int64 for 0 <= e < 2^27 (a kinetic-energy term),
// with one 32-bit conversion: e = 16 h + r with h = floor(e / 16) (exact; e / 16
// + 2^23 rounded toward -inf is 2^23 + h) and r in [0, 16) formed exactly by
// one fused multiply-add (r is a multiple of ulp(e) below 16); then
// e 2^28 = h 2^32 + r 2^28 and r 2^28 < 2^32 rounds within the low word.
// Identical to qfix<28>(e) on that range.
__device__ __forceinline__ long long q28_nonneg(float e)
{
    const float hm = __fadd_rd(__fmul_rn(e, 0.0625f), 8388608.0f);
    const int h = __float_as_int(hm) - 0x4B000000;
    const float r = __fmaf_rn(-16.0f, __fsub_rn(hm, 8388608.0f), e);
    const unsigned lo = __float2uint_rn(__fmul_rn(r, 268435456.0f));
    return (long long)(((unsigned long long)(unsigned)h << 32) | lo);
}

template <int RULE>
__device__ __forceinline__ void record_terms(float m, float vx, float vy, float vz, const float *xi, bool site,
                                             long long (&w)[MAX_WORDS32])
{
    const float px = __fmul_rn(m, vx), py = __fmul_rn(m, vy), pz = __fmul_rn(m, vz);
    w[0] = q32(px) + (site ? 0LL : COUNT48);
    w[1] = q32(py) + (site ? COUNT48 : 0LL);
    w[2] = q32(pz);
    if (RULE == 0) {
        const float e = __fadd_rn(__fadd_rn(__fmul_rn(px, vx), __fmul_rn(py, vy)), __fmul_rn(pz, vz));
        w[3] = q28_nonneg(e);
        w[4] = w[5] = 0;
    } else {
        w[3] = q32(__fmul_rn(m, xi[0]));
        w[4] = q32(__fmul_rn(m, xi[1]));
        w[5] = q32(__fmul_rn(m, xi[2]));
    }
}

// a count|momentum word: the signed low 48 bits and the high 16-bit count
__device__ __forceinline__ void unpack48(long long w, long long &count, long long &lo)
{
    lo = (long long)((unsigned long long)w << 16) >> 16;
    count = (long long)((unsigned long long)(w - lo) >> 48);
}

// split a pair word into its signed 32-bit halves
__device__ __forceinline__ void unpack2(long long w, long long &hi, long long &lo)
{
    lo = (long long)(int)(unsigned)(w & 0xFFFFFFFFll);
    hi = (w - lo) >> 32;
}

// uint64 / int64 -> float (rounded twice, |error| <= 1 ulp) without the 64-bit
// convert: the magnitude is split into 20 + 22 + 22 bits, each converted
// exactly, and the sign applied last (no cancellation between the pieces)
__device__ __forceinline__ float ull2f(unsigned long long w)
{
    const uint32_t h = (uint32_t)(w >> 44), m = (uint32_t)(w >> 22) & 0x3FFFFFu, l = (uint32_t)w & 0x3FFFFFu;
    const float hf = __uint_as_float(0x4B000000u | h) - 8388608.0f;   // exact for h < 2^23
    const float mf = __uint_as_float(0x4B000000u | m) - 8388608.0f;
    const float lf = __uint_as_float(0x4B000000u | l) - 8388608.0f;
    return fmaf(hf, 17592186044416.0f, fmaf(mf, 4194304.0f, lf));    // h 2^44 + m 2^22 + l
}
__device__ __forceinline__ float ll2f(long long w)
{
    return w < 0 ? -ull2f(0ull - (unsigned long long)w) : ull2f((unsigned long long)w);
}

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the kernel translation units).
// ---------------------------------------------------------------------------
enum : int { SOLV_COLLIDE = 1, SOLV_STREAM = 2, SOLV_BIN = 4 };

struct LaunchCfg {
    int block;      // threads per CTA of the solvent pass
    int grid;       // CTAs (persistent over tiles)
    int staged;     // 1: tiles staged through shared memory by bulk async copies
    int cap;        // particles per shared-memory stage (>= the tile size)
};

// solvent pass (kernels_solvent.cu)
void launch_solvent(const StepArgs &a, int flags, LaunchCfg cfg, cudaStream_t s);
void launch_params(const StepArgs &a, int grid, cudaStream_t s);
size_t solvent_stage_bytes(int precision, int rule, int cap);
size_t solvent_smem_bytes(int precision, int rule, int cap, int block);  // dynamic smem of the staged pass
void launch_aos_to_soa(const StepArgs &a, const void *xaos, const void *vaos, cudaStream_t s);
void launch_soa_to_aos(const StepArgs &a, void *xaos, void *vaos, const int64_t *out_off,
                       cudaStream_t s);
void launch_solvent_diag(const StepArgs &a, double *acc, cudaStream_t s);
// re-sort (kernels_solvent.cu)
void launch_sort_count(const StepArgs &a, int32_t *counts, int num_sms, cudaStream_t s);
void launch_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *block_sums, cudaStream_t s);

// Per-body velocity autocorrelation accumulators (translational and angular).
struct VacfArgs {
    int32_t n_lags, every;
    int64_t start;                       // completed steps when the accumulation began
    double *ring_v, *ring_w;             // [n_bodies][n_lags][3] last samples of V and omega
    double *ct, *cr;                     // [n_bodies][n_lags] sums of V(t).V(t+k), omega(t).omega(t+k)
    long long *count;                    // [n_lags] origins summed per lag
};
// after the POST coupling of a step, before the counter advances
void launch_vacf_sample(const StepArgs &a, const VacfArgs &g, cudaStream_t s);

// Reverse non-equilibrium momentum exchange between two slabs (replica 0).
constexpr int RN_BUCKETS = 512;    // rank-key histogram: 1/8-octave buckets from 2^-40 to 2^24,
                                   // smaller keys in the first, larger in the last
constexpr int RN_CAP = 4096;       // candidates kept per slab (MPCD_RNEMD_MAX_CANDIDATES)
constexpr int RN_LIST = 1 << 20;   // slab members listed per slab (MPCD_RNEMD_MAX_SLAB)
struct RnEntry {
    unsigned long long key;          // bits of the non-negative rank key (float or double)
    uint32_t tag, idx;               // particle id, slot - solv_begin
};
struct RnemdArgs {
    float ya0f, ya1f, yb0f, yb1f, vtf;   // slab bounds and target (P32 decisions)
    double ya0, ya1, yb0, yb1, vt;       // the same in double (P64 decisions)
    int32_t max_pairs, period;
    int32_t step_offset;                 // added to *d_step: the step whose collision follows
    int32_t fix_sums;                    // the solvent is already binned: correct its cell words
    int32_t *hist;                       // [2][RN_BUCKETS], zero between exchanges
    int32_t *count;                      // [2] slab members listed, zero between exchanges
    RnEntry *list;                       // [2][RN_LIST] slab members
    int32_t *ncand;                      // [2] candidates kept, zero between exchanges
    RnEntry *cand;                       // [2][RN_CAP] candidates
    double *p_total;                     // exchanged x momentum, A -> B
    long long *n_total;                  // exchanged pairs
};
// slab_members: the expected members of one slab (sizes the scan grid)
void launch_rnemd(const StepArgs &a, const RnemdArgs &g, int num_sms, int64_t slab_members, cudaStream_t s);
size_t rnemd_swap_smem();
// mass and momentum profile of replica 0 (solvent and bodies), FP64 [n_bins] each
void launch_velocity_profile(const StepArgs &a, int bin_axis, int vel_axis, int n_bins, double *mass, double *mom,
                             int num_sms, cudaStream_t s);
// re-sort by rank (perm[slot] = row in the replica) and gather into d, dtag
void launch_sort_rank_gather(const StepArgs &a, const int32_t *ex, const int32_t *counts, int32_t *cursor,
                             uint32_t *perm, void *const d[6], uint32_t *dtag, bool shifted, int num_sms,
                             cudaStream_t s);
// counts[c] = solvent members of cell c from the FP32 form's cell word 0
void launch_counts_from_words(int64_t C, const void *sums, int32_t *counts, int num_sms, cudaStream_t s);
void launch_sort_canonical(const StepArgs &a, void *const arr[6], uint32_t *tag,
                           const int32_t *offsets, cudaStream_t s);
size_t scan_block_sums_size(int64_t n);
// canonical member order of the collision at *d_step (counting sort by cell:
// histogram, scan, scatter, per-cell order solvent before sites, ascending id);
// counts and ex hold n_cells + 1 entries, keys and order n_solvent + n_sites
void launch_cell_order(const StepArgs &a, int64_t n_solvent, int32_t *counts, int32_t *ex, int32_t *cursor,
                       int32_t *scan_bs, unsigned long long *keys, int64_t *order, int64_t *start, int num_sms,
                       cudaStream_t s);

// host-state ingest / egress by stable radix sort (kernels_sort.cu)
size_t radix_hist_ints(int64_t n);          // ints of the per-pass digit histogram
int key_bits(uint64_t max_key);             // bits needed for keys <= max_key
// stable sort of (key, value) pairs by the low nbits; returns 1 if the result
// is in (kB, vB), 0 if in (kA, vA)
int launch_radix_sort(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, int64_t n, int nbits,
                      int32_t *hist, int32_t *hist_ex, int32_t *scan_bs, int *err, cudaStream_t s);
void launch_keys_in(const StepArgs &a, const void *xa, uint32_t *keys, uint32_t *vals, int64_t nslots,
                    cudaStream_t s);
// host rows -> 8-word records rec[n_rows][8] (the ingest gather reads one record per particle)
void launch_pack_rows(const StepArgs &a, const void *xa, const void *va, void *rec, int64_t n_rows, int num_sms,
                      cudaStream_t s);
void launch_gather_in(const StepArgs &a, const void *rec, const uint32_t *vals, int64_t nslots, int64_t n_rows,
                      int num_sms, cudaStream_t s);
void launch_keys_out(const StepArgs &a, uint32_t *keys, uint32_t *vals, int64_t nslots, uint32_t n_rows,
                     cudaStream_t s);
// slots -> records rec[nslots][8]; then the host rows [row0, row1) in order
// from them (vals[row] = the row's slot)
void launch_pack_slots(const StepArgs &a, void *rec, int64_t nslots, int num_sms, cudaStream_t s);
void launch_gather_rows(const StepArgs &a, const uint32_t *vals, const void *rec, void *xa, void *va, int64_t row0,
                        int64_t row1, int64_t nslots, int num_sms, cudaStream_t s);

// angular-momentum-conserving collision variants (kernels_angular.cu for the
// solvent and the per-cell solve, kernels_bodies.cu for the sites).
// Cell words, SoA [ANG_WORDS][n_cells], int64 (P32) or double (P64); Q is a
// member's integer lattice offset inside its shifted cell (units 2^-20), P its
// momentum term (P32: round(fl32(m v) 2^20); P64: m v):
enum : int { AW_COUNT = 0,      // 1 per solvent particle, 2^12 per site
             AW_SQ = 1,         // 1-3   sum Q of the solvent
             AW_SQB = 4,        // 4-6   sum Q of the sites
             AW_QQ = 7,         // 7-12  sum Q_a Q_b of the solvent (xx, yy, zz, xy, xz, yz)
             AW_QQB = 13,       // 13-18 the same of the sites
             AW_L = 19,         // 19-21 sum Q x (P - P*)
             AW_P = 22,         // 22-24 sum (P - P*)
             ANG_WORDS = 25 };
enum : int { ANG_PRE = 0, ANG_POST = 1, ANG_PARAMS = 2, ANG_APPLY = 3 };

// Per-cell record of the correction: the mass-weighted lattice sums sw = sum mu Q,
// the cell mass M = sum mu (mu = round(m 2^24) in P32, m in P64) and
// w' = w / (M 2^20); a member's offset from the centre of mass is (M Q - sw),
// an exact integer in P32 (|.| < M 2^20 < 2^63 for cell masses below 2^19).
template <typename Real> struct AngParams;
template <> struct AngParams<float> { long long sw[3]; long long M; float w[3]; float pad; };
template <> struct AngParams<double> { double sw[3]; double M; double w[3]; double pad; };

__device__ __forceinline__ int ang_lattice_q(float x, int S) { return (__float2int_rd(x * 1048576.0f) - S) & 0xFFFFF; }
__device__ __forceinline__ int ang_lattice_q(double x, int S) { return (__double2int_rd(x * 1048576.0) - S) & 0xFFFFF; }
__device__ __forceinline__ float ang_offset(const AngParams<float> &p, int Q, int k)
{
    return ll2f(p.M * (long long)Q - p.sw[k]);
}
__device__ __forceinline__ double ang_offset(const AngParams<double> &p, int Q, int k)
{
    return p.M * (double)Q - p.sw[k];
}
// v += w' x (M Q - sw) for a member with lattice offset Q
template <typename Real>
__device__ __forceinline__ void ang_correct(const AngParams<Real> &p, const int (&Q)[3], Real (&v)[3])
{
    const Real rc[3] = {ang_offset(p, Q[0], 0), ang_offset(p, Q[1], 1), ang_offset(p, Q[2], 2)};
    v[0] = v[0] + (p.w[1] * rc[2] - p.w[2] * rc[1]);
    v[1] = v[1] + (p.w[2] * rc[0] - p.w[0] * rc[2]);
    v[2] = v[2] + (p.w[0] * rc[1] - p.w[1] * rc[0]);
}
__device__ __forceinline__ void ang_red(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
__device__ __forceinline__ void ang_red(double *p, double v) { atomicAdd(p, v); }
template <typename Real> struct AngWord;
template <> struct AngWord<float> { typedef long long type; };
template <> struct AngWord<double> { typedef double type; };

size_t angular_param_bytes(int precision);
// solvent phases and the per-cell solve; ANG_PRE also writes a.ang_shift
void launch_angular(const StepArgs &a, int phase, int num_sms, cudaStream_t s);
// the sites' sums (ANG_PRE: thermalised velocities; ANG_POST: the rule's velocities);
// the correction itself is applied by the site POST coupling when a.ang_params is set
void launch_angular_sites(const StepArgs &a, int phase, cudaStream_t s);

// spatial domain decomposition into slabs (kernels_slab.cu); a.tiles are the
// fixed 2048-particle io tiles over the active particles
void launch_slab_count(const StepArgs &a, int zlo, int zhi, int32_t *leave, cudaStream_t s);
void launch_slab_split(const StepArgs &a, int zlo, int zhi, const int32_t *leave_ex, void *const dst[6],
                       uint32_t *dst_tag, void *const exp[6], uint32_t *exp_tag, cudaStream_t s);
void launch_slab_put(const StepArgs &a, const void *xa, const void *va, const uint32_t *tags, int64_t n, int64_t at,
                     int num_sms, cudaStream_t s);
void launch_slab_pack(int precision, void *const exp[6], const uint32_t *exp_tag, int64_t n, void *xa, void *va,
                      uint32_t *tags, int num_sms, cudaStream_t s);
void launch_words_add(int precision, void *sums, int nw, int64_t C, int64_t cell0, int64_t ncell, const void *add,
                      int num_sms, cudaStream_t s);
void launch_body_partial(const StepArgs &a, double *out, cudaStream_t s);
void launch_body_apply(const StepArgs &a, const double *dpl, cudaStream_t s);

// bodies and sites (kernels_bodies.cu)
void launch_body_md(const StepArgs &a, cudaStream_t s);
void launch_body_force(const StepArgs &a, int kick, cudaStream_t s);
void launch_sites_pre(const StepArgs &a, int max_sites, cudaStream_t s);
void launch_sites_post(const StepArgs &a, int max_sites, cudaStream_t s);
void launch_advance_step(const StepArgs &a, cudaStream_t s);
void launch_body_diag(const StepArgs &a, double *acc, cudaStream_t s);
void launch_body_impulse(const StepArgs &a, cudaStream_t s);
cudaError_t configure_body_kernels(int max_sites, int precision);

}  // namespace mpcd
