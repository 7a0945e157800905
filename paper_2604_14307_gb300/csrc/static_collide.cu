// mpcd_collide_solvent_static: one solvent collision (Sec. II.A) of a single
// periodic box whose scratch - cell sums, collision parameters, the work-tile
// tables, the step counter and the error word - lives in one statically
// reserved device array of this translation unit, so the call allocates no
// device memory.  The binning, parameter and collision kernels are the
// library's own (kernels_solvent.cu); only their scratch pointers differ from
// a context's.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <stdio.h>

#include "mpcd.h"
#include "mpcd_internal.cuh"

using namespace mpcd;

namespace {

constexpr int64_t MAX_CELLS = MPCD_STATIC_MAX_CELLS;
constexpr int64_t MAX_SOLVENT = MPCD_STATIC_MAX_SOLVENT;
constexpr int64_t TILE = 2048;                 // particles per work tile (a multiple of 4)
constexpr int64_t CELL_TILE = 256;             // cells per parameter tile (one CTA each)
constexpr int64_t MAX_TILES = MAX_SOLVENT / TILE;
constexpr int64_t MAX_CTILES = MAX_CELLS / CELL_TILE;
constexpr int MAX_WORDS = MAX_WORDS32;         // P32 cell words: 4 (SRD) or 6 (AT)

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_SUMS = 0;
constexpr size_t OFF_PARAMS = OFF_SUMS + align256(sizeof(long long) * MAX_WORDS * MAX_CELLS);
constexpr size_t OFF_TILES = OFF_PARAMS + align256(32 * MAX_CELLS);
constexpr size_t OFF_CTILES = OFF_TILES + align256(sizeof(Tile) * MAX_TILES);
constexpr size_t OFF_REP = OFF_CTILES + align256(sizeof(Tile) * MAX_CTILES);
constexpr size_t OFF_STEP = OFF_REP + align256(sizeof(DevReplica));
constexpr size_t OFF_ERR = OFF_STEP + 256;
constexpr size_t SCRATCH_BYTES = OFF_ERR + 256;

}  // namespace

// The whole scratch of the call (about 5.2 MB), reserved in the module image.
static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

namespace {

struct DeviceSetup {
    unsigned char *base = nullptr;
    int num_sms = 0;
};
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
DeviceSetup g_setup[MAX_DEVICES];

// Per-call initialisation of the scratch: replica record, regular tile
// tables, step counter, cleared error word and zeroed cell sums (the binning
// pass accumulates into them).
__global__ void k_static_setup(unsigned char *base, DevReplica rep, int64_t n_solvent, int64_t n_cells,
                               int n_words, int64_t step)
{
    long long *sums = reinterpret_cast<long long *>(base + OFF_SUMS);
    Tile *tiles = reinterpret_cast<Tile *>(base + OFF_TILES);
    Tile *ctiles = reinterpret_cast<Tile *>(base + OFF_CTILES);
    const int64_t n_tiles = (n_solvent + TILE - 1) / TILE;
    const int64_t n_ctiles = (n_cells + CELL_TILE - 1) / CELL_TILE;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < (int64_t)n_words * n_cells; i += stride) sums[i] = 0;
    for (int64_t t = t0; t < n_tiles; t += stride)
        tiles[t] = Tile{0, 0, t * TILE, min((t + 1) * TILE, n_solvent)};
    for (int64_t t = t0; t < n_ctiles; t += stride)
        ctiles[t] = Tile{0, 0, t * CELL_TILE, min((t + 1) * CELL_TILE, n_cells)};
    if (t0 == 0) {
        *reinterpret_cast<DevReplica *>(base + OFF_REP) = rep;
        *reinterpret_cast<int64_t *>(base + OFF_STEP) = step;
        *reinterpret_cast<int *>(base + OFF_ERR) = 0;
    }
}

int reject(char *msg, size_t len, const char *text)
{
    if (msg && len) snprintf(msg, len, "%s", text);
    return MPCD_ERR_ARG;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" int mpcd_collide_solvent_static(const mpcd_params *p, const int32_t L[3], int64_t n,
                                           const float *x, const float *y, const float *z, float *vx,
                                           float *vy, float *vz, const uint32_t *tag, int64_t step,
                                           void *stream, char *msg, size_t msg_len)
{
    char buf[160];
    if (!p || !L) return reject(msg, msg_len, "params and L must not be NULL");
    if (p->precision != MPCD_P32)
        return reject(msg, msg_len, "only the P32 form (FP32 state, fixed-point cell sums) is supported");
    if (p->rule != MPCD_SRD && p->rule != MPCD_AT) return reject(msg, msg_len, "rule must be MPCD_SRD or MPCD_AT");
    if (!(p->kT > 0.0) || !(p->m_solvent > 0.0) || !(p->alpha_deg == p->alpha_deg) ||
        p->thermostat < 0 || p->thermostat > 2 || p->angular != 0)
        return reject(msg, msg_len, "invalid params (kT > 0, m_solvent > 0, thermostat 0/1/2, angular 0)");
    // the binning rule forms floor(x 2^20) in 32 bits, so an edge must stay below 2048 cells
    if (L[0] < 3 || L[1] < 3 || L[2] < 3 || L[0] > 2047 || L[1] > 2047 || L[2] > 2047)
        return reject(msg, msg_len, "every box edge L must be 3 to 2047 cells");
    const int64_t cells = (int64_t)L[0] * L[1] * L[2];
    if (cells > MAX_CELLS) {
        snprintf(buf, sizeof buf, "box of %lld cells exceeds the static scratch limit of %lld cells",
                 (long long)cells, (long long)MAX_CELLS);
        return reject(msg, msg_len, buf);
    }
    if (n < 0 || n > MAX_SOLVENT) {
        snprintf(buf, sizeof buf, "n_solvent %lld outside [0, %lld]", (long long)n, (long long)MAX_SOLVENT);
        return reject(msg, msg_len, buf);
    }
    if (n % 4 != 0) return reject(msg, msg_len, "n_solvent must be a multiple of 4");
    if (step < 0) return reject(msg, msg_len, "step must be >= 0");
    if (n > 0) {
        if (!x || !y || !z || !vx || !vy || !vz) return reject(msg, msg_len, "solvent arrays must not be NULL");
        if (p->rule == MPCD_AT && !tag) return reject(msg, msg_len, "MPCD_AT needs the tag array");
        if (!aligned16(x) || !aligned16(y) || !aligned16(z) || !aligned16(vx) || !aligned16(vy) ||
            !aligned16(vz) || (tag && !aligned16(tag)))
            return reject(msg, msg_len, "device arrays must be 16-byte aligned");
    }
    if (msg && msg_len) msg[0] = 0;
    if (n == 0) return MPCD_OK;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return reject(msg, msg_len, "no usable current CUDA device");
    }
    DeviceSetup su;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_setup[dev].base) {
            void *addr = nullptr;
            int sms = 0;
            if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                if (msg && msg_len) snprintf(msg, msg_len, "static scratch lookup failed");
                return MPCD_ERR_CUDA;
            }
            g_setup[dev].base = static_cast<unsigned char *>(addr);
            g_setup[dev].num_sms = sms;
        }
        su = g_setup[dev];
    }

    const int nw = p->rule == MPCD_SRD ? Words32<0>::n : Words32<1>::n;
    DevReplica rep{};
    rep.L[0] = L[0]; rep.L[1] = L[1]; rep.L[2] = L[2];
    rep.cell_base = 0;
    rep.solv_begin = 0;
    rep.n_solvent = n;
    rep.site_id_base = n;
    rep.body_begin = rep.body_end = 0;
    rep.site_begin = 0;
    rep.row_begin = 0;
    rep.key0 = (uint32_t)p->seed;
    rep.key1 = (uint32_t)(p->seed >> 32);   // replica 0: seed_hi ^ 0

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_tiles = (n + TILE - 1) / TILE;
    const int64_t n_ctiles = (cells + CELL_TILE - 1) / CELL_TILE;
    const int64_t setup_work = std::max<int64_t>((int64_t)nw * cells, n_tiles);
    const int setup_grid = (int)std::min<int64_t>((setup_work + 255) / 256, (int64_t)su.num_sms * 4);
    k_static_setup<<<setup_grid, 256, 0, s>>>(su.base, rep, n, cells, nw, step);

    StepArgs a{};
    a.precision = MPCD_P32;
    a.rule = p->rule;
    a.thermostat = p->thermostat;
    a.naive = 0;
    a.kT = p->kT;
    a.dt = p->dt;
    a.m_solvent = p->m_solvent;
    const double al = p->alpha_deg * 3.14159265358979323846264338327950288 / 180.0;
    a.cos_a = std::cos(al);
    a.sin_a = std::sin(al);
    a.kTf = (float)p->kT;
    a.dtf = (float)p->dt;
    a.m_solvent_f = (float)p->m_solvent;
    a.cos_af = (float)a.cos_a;
    a.sin_af = (float)a.sin_a;
    a.qm_solvent = (long long)std::llrint((double)a.m_solvent_f * 16777216.0);
    a.m_site_f = 0.0f;
    a.qm_site = 0;
    a.reps = reinterpret_cast<const DevReplica *>(su.base + OFF_REP);
    a.n_rep = 1;
    a.tiles = reinterpret_cast<const Tile *>(su.base + OFF_TILES);
    a.n_tiles = (int32_t)n_tiles;
    a.ctiles = reinterpret_cast<const Tile *>(su.base + OFF_CTILES);
    a.n_ctiles = (int32_t)n_ctiles;
    a.x = const_cast<float *>(x);
    a.y = const_cast<float *>(y);
    a.z = const_cast<float *>(z);
    a.vx = vx;
    a.vy = vy;
    a.vz = vz;
    a.tag = const_cast<uint32_t *>(tag);
    a.sums = su.base + OFF_SUMS;
    a.params = su.base + OFF_PARAMS;
    a.dbg_sums = nullptr;
    a.n_cells = cells;
    a.nw = nw;
    a.d_step = reinterpret_cast<const int64_t *>(su.base + OFF_STEP);
    a.d_err = reinterpret_cast<int *>(su.base + OFF_ERR);

    // direct (unstaged) passes: bin at the step's shift, per-cell parameters,
    // then the collision of every particle (the order of mpcd_collide)
    const LaunchCfg cfg{256, (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)su.num_sms * 4)), 0,
                        (int)TILE};
    launch_solvent(a, SOLV_BIN, cfg, s);
    launch_params(a, 0, s);
    launch_solvent(a, SOLV_COLLIDE, cfg, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (msg && msg_len) snprintf(msg, msg_len, "launch failed: %s", cudaGetErrorString(e));
        return MPCD_ERR_CUDA;
    }
    return MPCD_OK;
}
