// C ABI of the MPCD + rigid-body library (include/mpcd.h): context, memory,
// launch orchestration, software pipelining of whole steps, periodic re-sort,
// CUDA-graph capture, per-kernel event timing and the autotuner.
#include "../../include/mpcd.h"
#include "mpcd_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using namespace mpcd;

namespace {

struct KStat {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};
struct Pending {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
};
struct GraphEntry {
    cudaGraphExec_t exec;
    int cur_end;
    int64_t since_end;
};

}  // namespace

struct mpcd_ctx {
    int device = 0;
    mpcd_params prm{};
    mpcd_allocator alloc{};
    bool use_alloc = false;
    int status = MPCD_OK;
    char err[512] = "ok";

    int nrep = 0, nshapes = 0, max_sites = 0;
    double max_wca_d = 0.0;
    double m_site = 0.0;   // the common site mass (required by the P32 form)
    int64_t Ns = 0, Nslots = 0, B = 0, Nsite = 0, C = 0;
    int nw = 0, realsz = 0, param_bytes = 0;
    std::vector<DevReplica> reps;
    std::vector<Tile> tiles, ctiles;
    std::vector<DevShape> shapes;

    std::vector<void *> allocations;
    int64_t dev_bytes = 0;
    DevReplica *d_reps = nullptr;
    Tile *d_tiles = nullptr, *d_ctiles = nullptr;
    int64_t tiles_cap = 0;
    // fixed 2048-particle tiles of the helper passes (sort, state I/O,
    // diagnostics), whatever tile size the solvent pass is tuned to
    std::vector<Tile> io_tiles;
    Tile *d_io_tiles = nullptr;
    DevShape *d_shapes = nullptr;
    DevBody *d_bodies = nullptr;
    float4 *d_bpos = nullptr, *d_bpos_build = nullptr;
    int32_t *d_nlist = nullptr, *d_ncount = nullptr;
    int *d_nl_dirty = nullptr;
    float *d_pose32 = nullptr;
    double *d_pose64 = nullptr;
    void *d_partial = nullptr;
    double *d_tb = nullptr, *d_tm = nullptr, *d_tcent = nullptr;
    double *d_cent64 = nullptr;                 // rotated WCA centres of every body
    float4 *d_cent32 = nullptr;
    int64_t n_cent_bodies = 0;                  // WCA centres over all bodies
    int max_cent = 0;                           // most centres of any shape
    float *d_tbf = nullptr, *d_tmf = nullptr;
    void *sol[2][6] = {};
    uint32_t *tag[2] = {nullptr, nullptr};
    int cur = 0;
    void *sums = nullptr, *params = nullptr, *dbg_sums = nullptr;
    bool debug = false;
    void *site_v = nullptr;
    int32_t *site_cell = nullptr;
    int64_t *d_step = nullptr;
    int *d_err = nullptr;
    int *d_tile_ctr = nullptr;      // work counter of the staged solvent pass
    double *d_diag = nullptr;
    int32_t *counts = nullptr, *ex = nullptr, *cursor = nullptr, *scan_bs = nullptr;
    int32_t *rs_hist = nullptr, *rs_ex = nullptr, *rs_bs = nullptr;   // radix-sort digit counts
    void *rec = nullptr;            // [Nslots][8] Real: particle records for the state permutations
    void *staging = nullptr;

    int64_t step = 0, since_sort = 0, last_key = -1;
    int num_sms = 0;
    mpcd_tuning tune{512, 2048, 1, 20, 2};
    int smem_per_sm = 0;

    bool profiling = false;
    std::vector<Pending> pending;
    std::map<std::string, KStat> prof;
    std::vector<cudaEvent_t> evpool;

    std::map<std::tuple<int64_t, int, int64_t>, GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t io_stream = nullptr;           // host copies that overlap with kernels
    cudaEvent_t io_ev[2] = {nullptr, nullptr};
    static constexpr int OUT_CHUNKS = 8;         // egress: row chunks gathered and copied in turn
    cudaEvent_t out_ev[OUT_CHUNKS + 1] = {};
    cudaStream_t side = nullptr;                // site/body chain beside the solvent pass
    cudaEvent_t side_ev[2] = {nullptr, nullptr};

    // reverse non-equilibrium exchange (allocated on first use)
    mpcd_rnemd rn{};
    int32_t *rn_hist = nullptr, *rn_count = nullptr;
    RnEntry *rn_list = nullptr, *rn_cand = nullptr;
    int32_t *rn_ncand = nullptr;
    double *rn_tot = nullptr;                   // [0] momentum, [1] pairs (as long long)
    double *d_profile = nullptr;                // [2][PROFILE bins] velocity-profile sums
    void *ang_words = nullptr;                  // [ANG_WORDS][C] angular-momentum sums (+a variants)
    void *ang_params = nullptr;                 // [C] AngParams records of the +a correction
    int4 *ang_shift = nullptr;                  // [nrep] grid shift of the current collision
    double f_ext[3] = {0.0, 0.0, 0.0};          // constant force on every body (one replica)
    VacfArgs vacf{};                            // velocity autocorrelations (n_lags 0: off)
    // slab of a decomposed box (mpcd_create_slab): the active solvent count is
    // reps[0].n_solvent (= Ns), the slots hold `capacity` particles
    bool slab = false;
    int32_t slab_zlo = 0, slab_zhi = 0;
    int64_t capacity = 0;
    void *exp_sol[6] = {};                       // the particles that left the slab
    uint32_t *exp_tag = nullptr;
    uint32_t *tag_stage = nullptr;               // ids of the particles in `staging`
    int64_t n_exp = 0;
    int32_t *slab_leave = nullptr, *slab_leave_ex = nullptr, *slab_bs = nullptr;
    double *d_dpl = nullptr;                     // [B][6] transfer of the slab's own sites
    void *words_stage = nullptr;                 // neighbour words to add
    int64_t words_stage_bytes = 0;
    // canonical member order (mpcd_cell_order; allocated on first use)
    int32_t *ord_counts = nullptr, *ord_ex = nullptr, *ord_cursor = nullptr, *ord_bs = nullptr;
    unsigned long long *ord_keys = nullptr;
    int64_t *ord_out = nullptr, *ord_start = nullptr;
    bool have_state = false;                    // mpcd_set_state has run
};

namespace {

void clear_graphs(mpcd_ctx *c);
int fail(mpcd_ctx *c, int st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(mpcd_ctx *c, int st, const char *fmt, ...)
{
    if (c && c->status == MPCD_OK) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
        c->status = st;
    }
    return st;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? MPCD_ERR_OOM : MPCD_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

#define CHECK_CTX(ctx)                         \
    do {                                       \
        if (!(ctx)) return MPCD_ERR_ARG;       \
        if ((ctx)->status) return (ctx)->status; \
    } while (0)

void *dalloc(mpcd_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c->use_alloc) {
        p = c->alloc.alloc(bytes, c->alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocations.push_back(p);
        c->dev_bytes += (int64_t)bytes;
    }
    return p;
}

StepArgs make_args(const mpcd_ctx *c)
{
    StepArgs a{};
    const mpcd_params &p = c->prm;
    a.precision = p.precision;
    a.rule = p.rule;
    a.thermostat = p.thermostat;
    a.naive = p.naive_transfer;
    a.kT = p.kT;
    a.dt = p.dt;
    a.m_solvent = p.m_solvent;
    double al = p.alpha_deg * 3.14159265358979323846264338327950288 / 180.0;
    a.cos_a = std::cos(al);
    a.sin_a = std::sin(al);
    a.kTf = (float)p.kT;
    a.dtf = (float)p.dt;
    a.m_solvent_f = (float)p.m_solvent;
    a.cos_af = (float)a.cos_a;
    a.sin_af = (float)a.sin_a;
    a.qm_solvent = (long long)std::llrint((double)a.m_solvent_f * 16777216.0);
    a.m_site_f = (float)c->m_site;
    a.m_site = c->m_site;
    a.ang_words = c->ang_words;
    a.ang_params = c->ang_params;
    a.ang_shift = c->ang_shift;
    a.qm_site = (long long)std::llrint((double)a.m_site_f * 16777216.0);
    a.reps = c->d_reps;
    a.n_rep = c->nrep;
    a.tiles = c->d_tiles;
    a.n_tiles = (int32_t)c->tiles.size();
    a.ctiles = c->d_ctiles;
    a.n_ctiles = (int32_t)c->ctiles.size();
    a.x = c->sol[c->cur][0];
    a.y = c->sol[c->cur][1];
    a.z = c->sol[c->cur][2];
    a.vx = c->sol[c->cur][3];
    a.vy = c->sol[c->cur][4];
    a.vz = c->sol[c->cur][5];
    a.tag = c->tag[c->cur];
    a.sums = c->sums;
    a.params = c->params;
    a.dbg_sums = c->debug ? c->dbg_sums : nullptr;
    a.n_cells = c->C;
    a.nw = c->nw;
    a.bodies = c->d_bodies;
    a.bpos = c->d_bpos;
    a.bpos_build = c->d_bpos_build;
    a.nlist = c->d_nlist;
    a.ncount = c->d_ncount;
    a.nl_dirty = c->d_nl_dirty;
    a.pose32 = c->d_pose32;
    a.pose64 = c->d_pose64;
    a.partial = c->d_partial;
    a.n_bodies = (int32_t)c->B;
    a.shapes = c->d_shapes;
    a.tb = c->d_tb;
    a.tbf = c->d_tbf;
    a.tm = c->d_tm;
    a.tmf = c->d_tmf;
    a.tcent = c->d_tcent;
    a.max_wca_d = c->max_wca_d;
    a.max_cent = c->max_cent;
    a.cent64 = c->d_cent64;
    a.cent32 = c->d_cent32;
    a.site_v = c->site_v;
    a.site_cell = c->site_cell;
    a.n_sites = c->Nsite;
    a.d_step = c->d_step;
    a.d_err = c->d_err;
    a.tile_ctr = c->d_tile_ctr;
    a.site_own = c->slab ? 1 : 0;
    a.site_zlo = c->slab_zlo;
    a.site_zhi = c->slab_zhi;
    // constant body force, balanced by a uniform force on the solvent of the
    // (single) replica: each particle gets -B f / N_s, i.e. acceleration g
    if (c->f_ext[0] != 0.0 || c->f_ext[1] != 0.0 || c->f_ext[2] != 0.0) {
        for (int k = 0; k < 3; ++k) {
            a.fext[k] = c->f_ext[k];
            const double g = -((double)c->B * c->f_ext[k]) / ((double)c->Ns * p.m_solvent);
            a.ah[k] = 0.5 * g * p.dt;
            a.ahf[k] = (float)a.ah[k];
        }
        a.accel = 1;
    }
    return a;
}

// arguments of the helper passes: the same as make_args but over the fixed
// 2048-particle tiles
StepArgs make_io_args(const mpcd_ctx *c)
{
    StepArgs a = make_args(c);
    a.tiles = c->d_io_tiles;
    a.n_tiles = (int32_t)c->io_tiles.size();
    return a;
}

void build_tiles(mpcd_ctx *c)
{
    c->tiles.clear();
    const int64_t T = c->tune.tile;   // a multiple of 8 (set_tuning rounds it)
    for (int r = 0; r < c->nrep; ++r) {
        const DevReplica &R = c->reps[r];
        for (int64_t b = R.solv_begin; b < R.solv_begin + R.n_solvent; b += T)
            c->tiles.push_back(Tile{r, 0, b, std::min(b + T, R.solv_begin + R.n_solvent)});
    }
}

void build_ctiles(mpcd_ctx *c)
{
    c->ctiles.clear();
    const int64_t T = 256;   // the parameter and canonical-sort kernels take one tile per CTA
    for (int r = 0; r < c->nrep; ++r) {
        const DevReplica &R = c->reps[r];
        int64_t n = (int64_t)R.L[0] * R.L[1] * R.L[2];
        for (int64_t b = R.cell_base; b < R.cell_base + n; b += T)
            c->ctiles.push_back(Tile{r, 0, b, std::min(b + T, (int64_t)R.cell_base + n)});
    }
}

int upload_tiles(mpcd_ctx *c)
{
    if ((int64_t)c->tiles.size() > c->tiles_cap) {
        c->tiles_cap = (int64_t)c->tiles.size() * 2 + 16;
        c->d_tiles = (Tile *)dalloc(c, c->tiles_cap * sizeof(Tile));
        if (!c->d_tiles) return fail(c, MPCD_ERR_OOM, "tile table allocation failed");
    }
    if (!c->tiles.empty())
        CK(c, cudaMemcpy(c->d_tiles, c->tiles.data(), c->tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    return MPCD_OK;
}

// the active solvent count of a slab context changed: replica record, work
// tiles of the solvent pass and of the helper passes, CUDA graphs
int slab_set_count(mpcd_ctx *c, int64_t n)
{
    c->reps[0].n_solvent = n;
    c->Ns = n;
    CK(c, cudaMemcpy(c->d_reps, c->reps.data(), c->reps.size() * sizeof(DevReplica), cudaMemcpyHostToDevice));
    build_tiles(c);
    int e = upload_tiles(c);
    if (e) return e;
    c->io_tiles.clear();
    const DevReplica &R = c->reps[0];
    for (int64_t b = R.solv_begin; b < R.solv_begin + R.n_solvent; b += 2048)
        c->io_tiles.push_back(Tile{0, 0, b, std::min<int64_t>(b + 2048, R.solv_begin + R.n_solvent)});
    if (!c->io_tiles.empty())
        CK(c, cudaMemcpy(c->d_io_tiles, c->io_tiles.data(), c->io_tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    clear_graphs(c);
    return MPCD_OK;
}

// ------------------------------------------------------------- profiling
template <typename F>
int timed(mpcd_ctx *c, const char *name, double bytes, cudaStream_t s, F &&launch)
{
    if (!c->profiling) {
        launch();
        return MPCD_OK;
    }
    cudaEvent_t e0, e1;
    if (c->evpool.size() >= 2) {
        e0 = c->evpool.back(); c->evpool.pop_back();
        e1 = c->evpool.back(); c->evpool.pop_back();
    } else {
        CK(c, cudaEventCreate(&e0));
        CK(c, cudaEventCreate(&e1));
    }
    CK(c, cudaEventRecord(e0, s));
    launch();
    CK(c, cudaEventRecord(e1, s));
    c->pending.push_back(Pending{name, e0, e1, bytes});
    return MPCD_OK;
}

int drain_profile(mpcd_ctx *c)
{
    for (auto &p : c->pending) {
        CK(c, cudaEventSynchronize(p.b));
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, p.a, p.b));
        KStat &k = c->prof[p.name];
        k.launches += 1;
        k.ms += ms;
        k.bytes = p.bytes;
        c->evpool.push_back(p.a);
        c->evpool.push_back(p.b);
    }
    c->pending.clear();
    return MPCD_OK;
}

// algorithmic bytes of one solvent pass (see the design notes)
double solvent_bytes(const mpcd_ctx *c, int flags)
{
    double n = (double)c->Ns, rs = c->realsz, C = (double)c->C;
    double b = 0;
    if (flags & SOLV_STREAM) b += 2 * 3 * rs * n;            // r read + write
    else if (flags & (SOLV_COLLIDE | SOLV_BIN)) b += 3 * rs * n;  // r read
    if (flags & SOLV_COLLIDE) b += 2 * 3 * rs * n + C * c->param_bytes;   // v read+write, params
    else if (flags & SOLV_BIN) b += 3 * rs * n;              // v read
    if (c->prm.rule == MPCD_AT) b += 4 * n;                    // tags
    if (flags & SOLV_BIN) b += C * c->nw * 8.0;              // sums written once
    return b;
}

// ----------------------------------------------------------- step pieces
// dynamic shared memory of the staged or warp-specialised solvent pass
// (three-stage rings)
size_t ring_bytes(const mpcd_ctx *c, int mode, int tile, int block)
{
    const size_t stage = solvent_stage_bytes(c->prm.precision, c->prm.rule, tile);
    if (mode == 3) return (size_t)(block / 32) * 3 * stage;   // one three-stage ring per warp
    return 3 * stage;
}

bool staged_fits(const mpcd_ctx *c, int tile, int mode, int block)
{
    if (mode == 3 && (block > 512 || block % 32)) return false;
    const size_t lim = (mode == 3 ? 220 : 200) * 1024;
    return ring_bytes(c, mode, tile, block) <= lim;
}

LaunchCfg solvent_cfg(const mpcd_ctx *c)
{
    const int mode =
        c->tune.staged && staged_fits(c, c->tune.tile, c->tune.staged, c->tune.block) ? c->tune.staged : 0;
    LaunchCfg cfg{c->tune.block, 1, mode, c->tune.tile};
    int per_sm = c->tune.ctas_per_sm;
    if (mode) {
        size_t bytes = ring_bytes(c, mode, c->tune.tile, c->tune.block) + 4096;
        per_sm = std::max(1, std::min<int>(per_sm, (int)(c->smem_per_sm / bytes)));
    }
    const int threads = c->tune.block + (mode == 2 ? 32 : 0);
    per_sm = std::max(1, std::min(per_sm, 2048 / threads));
    cfg.grid = std::max(1, std::min((int)c->tiles.size(), c->num_sms * per_sm));
    return cfg;
}

int k_stream(mpcd_ctx *c, cudaStream_t s)
{
    StepArgs a = make_args(c);
    LaunchCfg cfg = solvent_cfg(c);
    int e = timed(c, "solvent_stream", solvent_bytes(c, SOLV_STREAM), s, [&] { launch_solvent(a, SOLV_STREAM, cfg, s); });
    if (e) return e;
    e = timed(c, "body_md", 0, s, [&] { launch_body_md(a, s); });
    if (e) return e;
    return timed(c, "body_force", 0, s, [&] { launch_body_force(a, 1, s); });
}

int k_bodies(mpcd_ctx *c, cudaStream_t s)
{
    StepArgs a = make_args(c);
    int e = timed(c, "body_md", 0, s, [&] { launch_body_md(a, s); });
    if (e) return e;
    return timed(c, "body_force", 0, s, [&] { launch_body_force(a, 1, s); });
}

int k_pre(mpcd_ctx *c, cudaStream_t s, int step_offset = 0)
{
    StepArgs a = make_args(c);
    a.step_offset = step_offset;
    double bytes = (double)c->Nsite * (3.0 * c->realsz + 4.0);
    return timed(c, "sites_pre", bytes, s, [&] { launch_sites_pre(a, c->max_sites, s); });
}

int k_params(mpcd_ctx *c, cudaStream_t s)
{
    StepArgs a = make_args(c);
    double bytes = (double)c->C * (2.0 * c->nw * 8.0 + c->param_bytes);
    return timed(c, "cell_params", bytes, s, [&] { launch_params(a, c->num_sms * 8, s); });
}

int k_post(mpcd_ctx *c, cudaStream_t s)
{
    StepArgs a = make_args(c);
    double bytes = (double)c->Nsite * (3.0 * c->realsz + 4.0);
    int e = timed(c, "sites_post", bytes, s, [&] { launch_sites_post(a, c->max_sites, s); });
    if (e) return e;
    return timed(c, "body_impulse", 0, s, [&] { launch_body_impulse(a, s); });
}

// velocity-autocorrelation sample after the POST coupling of a step
int k_vacf(mpcd_ctx *c, cudaStream_t s)
{
    if (c->vacf.n_lags == 0 || c->B == 0) return MPCD_OK;
    StepArgs a = make_args(c);
    return timed(c, "vacf", 0, s, [&] { launch_vacf_sample(a, c->vacf, s); });
}

int k_solvent(mpcd_ctx *c, int flags, cudaStream_t s)
{
    StepArgs a = make_args(c);
    LaunchCfg cfg = solvent_cfg(c);
    const char *name = flags == (SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN) ? "solvent_fused"
                       : flags == SOLV_COLLIDE                          ? "solvent_collide"
                       : flags == SOLV_BIN                              ? "solvent_bin"
                       : flags == (SOLV_STREAM | SOLV_BIN)              ? "solvent_stream_bin"
                                                                        : "solvent_stream";
    return timed(c, name, solvent_bytes(c, flags), s, [&] { launch_solvent(a, flags, cfg, s); });
}

int k_advance(mpcd_ctx *c, cudaStream_t s)
{
    StepArgs a = make_args(c);
    launch_advance_step(a, s);
    c->last_key = c->step;
    c->step += 1;
    return MPCD_OK;
}

static_assert(RN_CAP == MPCD_RNEMD_MAX_CANDIDATES, "candidate capacity of the exchange");
static_assert(RN_LIST == MPCD_RNEMD_MAX_SLAB, "slab capacity of the exchange");

// the exchange before the collision of step *d_step + step_offset; fix: the
// solvent is already binned for that collision
int k_rnemd(mpcd_ctx *c, cudaStream_t s, int step_offset, int fix)
{
    if (!c->rn.enabled || c->Ns == 0) return MPCD_OK;
    StepArgs a = make_args(c);
    RnemdArgs g{};
    const mpcd_rnemd &r = c->rn;
    g.ya0 = r.y_a; g.ya1 = r.y_a + r.width; g.yb0 = r.y_b; g.yb1 = r.y_b + r.width; g.vt = r.v_target;
    g.ya0f = (float)g.ya0; g.ya1f = (float)g.ya1; g.yb0f = (float)g.yb0; g.yb1f = (float)g.yb1;
    g.vtf = (float)g.vt;
    g.max_pairs = r.max_pairs;
    g.period = r.period;
    g.step_offset = step_offset;
    g.fix_sums = fix;
    g.hist = c->rn_hist;
    g.count = c->rn_count;
    g.list = c->rn_list;
    g.ncand = c->rn_ncand;
    g.cand = c->rn_cand;
    g.p_total = c->rn_tot;
    g.n_total = reinterpret_cast<long long *>(c->rn_tot + 1);
    const int64_t members = (int64_t)std::ceil((double)c->Ns * r.width / (double)c->reps[0].L[1]);
    return timed(c, "rnemd", 0, s, [&] { launch_rnemd(a, g, c->num_sms, members, s); });
}

// Counting sort of the solvent by cell.  from_words (the pipelined step, FP32
// form, after the solvent pass has binned every particle for the next
// collision): the cells are those of the next collision and their solvent
// counts are read from the cell words, so the count pass is skipped; else the
// unshifted cells, counted.  The order changes no result.
int do_sort(mpcd_ctx *c, int canonical, cudaStream_t s, bool from_words = false)
{
    if (c->Ns == 0) return MPCD_OK;
    StepArgs a = make_io_args(c);
    const int nxt = c->cur ^ 1;
    const bool words = from_words && !canonical && c->prm.precision == MPCD_P32;
    // algorithmic bytes: positions read by the count and rank passes (or the
    // count words), the source index written and read, the state and tags read
    // and written once
    double bytes = (double)c->Ns * (3.0 * c->realsz + 2.0 * 4.0 + 2.0 * (6.0 * c->realsz + 4.0)) +
                   (words ? (double)c->C * (8.0 + 4.0) : (double)c->Ns * 3.0 * c->realsz);
    int e = timed(c, "sort", bytes, s, [&] {
        cudaMemsetAsync(c->cursor, 0, c->C * sizeof(int32_t), s);
        cudaMemsetAsync(c->tag[nxt], 0xFF, c->Nslots * sizeof(uint32_t), s);
        if (words) {
            launch_counts_from_words(c->C, c->sums, c->counts, c->num_sms, s);
        } else {
            cudaMemsetAsync(c->counts, 0, c->C * sizeof(int32_t), s);
            launch_sort_count(a, c->counts, c->num_sms, s);
        }
        launch_scan(c->counts, c->ex, c->C, c->scan_bs, s);
        void *dst[6] = {c->sol[nxt][0], c->sol[nxt][1], c->sol[nxt][2],
                        c->sol[nxt][3], c->sol[nxt][4], c->sol[nxt][5]};
        // the permutation lives in the state-transfer record buffer (unused
        // between state transfers; Nslots x 32 bytes)
        launch_sort_rank_gather(a, c->ex, c->counts, c->cursor, (uint32_t *)c->rec, dst, c->tag[nxt], words,
                                c->num_sms, s);
        if (canonical) launch_sort_canonical(a, dst, c->tag[nxt], c->ex, s);
    });
    if (e) return e;
    c->cur = nxt;
    c->since_sort = 0;
    return MPCD_OK;
}

// one pass of the +a correction (kernels_angular.cu; the sites' sums in
// kernels_bodies.cu)
int k_ang(mpcd_ctx *c, int phase, cudaStream_t s)
{
    static const char *names[] = {"angular_pre", "angular_post", "angular_params", "angular_apply"};
    // algorithmic bytes: the solvent arrays each pass reads (and writes), the
    // cell words written or read once, the per-cell records
    const double N = (double)c->Ns, C = (double)c->C, r = c->realsz;
    const double rec = (double)angular_param_bytes(c->prm.precision);
    const double bytes[] = {N * 6 * r + C * 16 * 8, N * 6 * r + C * 6 * 8,
                            C * (2.0 * ANG_WORDS * 8 + rec), N * 9 * r + C * rec};
    StepArgs a = make_args(c);
    int e = timed(c, names[phase], bytes[phase], s, [&] { launch_angular(a, phase, c->num_sms, s); });
    if (!e && c->B > 0 && (phase == ANG_PRE || phase == ANG_POST)) {
        const double sb = (double)c->Nsite * (3.0 * r + 4.0);
        e = timed(c, phase == ANG_PRE ? "angular_sites_pre" : "angular_sites_post", sb, s,
                  [&] { launch_angular_sites(a, phase, s); });
    }
    return e;
}

// the unpipelined collision of the solvent at the current step (a2, a5-a7):
// exchange, binning, cell parameters, rule; with the +a variant the angular
// sums are taken before and after the rule and the correction applied
int k_collide(mpcd_ctx *c, cudaStream_t s)
{
    const bool ang = c->prm.angular != 0;
    int e = k_rnemd(c, s, 0, 0);
    if (!e) e = k_solvent(c, SOLV_BIN, s);
    if (!e && ang) e = k_ang(c, ANG_PRE, s);
    if (!e) e = k_params(c, s);
    if (!e) e = k_solvent(c, SOLV_COLLIDE, s);
    if (!e && ang) e = k_ang(c, ANG_POST, s);
    if (!e && ang) e = k_ang(c, ANG_PARAMS, s);
    if (!e && ang) e = k_ang(c, ANG_APPLY, s);
    return e;
}

// whole steps in the unpipelined order stream, couple(PRE), collide,
// couple(POST) (the +a variants, whose correction needs the cell totals of
// the rule's velocities before any particle streams on)
int run_steps_unfused(mpcd_ctx *c, int64_t n, cudaStream_t s)
{
    int e = MPCD_OK;
    for (int64_t k = 0; k < n && !e; ++k) {
        if ((e = k_stream(c, s))) break;
        if ((e = k_pre(c, s))) break;
        if ((e = k_collide(c, s))) break;
        if ((e = k_post(c, s))) break;
        if ((e = k_vacf(c, s))) break;
        if ((e = k_advance(c, s))) break;
        if (c->prm.sort_period >= 0 && ++c->since_sort >= c->tune.sort_period)
            if ((e = do_sort(c, 0, s))) break;
    }
    if (!e && !c->profiling) {
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(c, MPCD_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(ce));
    }
    return e;
}

// whole steps, software-pipelined: the solvent pass of step k collides (k),
// streams and bins for step k+1; beside it, on a second stream, run the site
// POST coupling of step k and the body step and site PRE coupling of step k+1
// (they need step k's cell parameters and impulse, not its solvent pass; both
// branches add to the cleared cell sums of step k+1 with integer atomics, so
// the order between them changes no result).  The branches join before the
// cell parameters of step k+1.
int run_steps(mpcd_ctx *c, int64_t n, cudaStream_t s)
{
    if (n <= 0) return MPCD_OK;
    if (c->prm.angular) return run_steps_unfused(c, n, s);
    int e = k_solvent(c, SOLV_STREAM | SOLV_BIN, s);
    if (!e) e = k_rnemd(c, s, 0, 1);
    if (!e) e = k_bodies(c, s);
    if (!e) e = k_pre(c, s);
    for (int64_t k = 0; k < n && !e; ++k) {
        if ((e = k_params(c, s))) break;
        if (k == n - 1) {
            if ((e = k_post(c, s))) break;
            if ((e = k_vacf(c, s))) break;
            if ((e = k_solvent(c, SOLV_COLLIDE, s))) break;
        } else {
            CK(c, cudaEventRecord(c->side_ev[0], s));
            CK(c, cudaStreamWaitEvent(c->side, c->side_ev[0], 0));
            if ((e = k_post(c, c->side))) break;
            if ((e = k_vacf(c, c->side))) break;
            if ((e = k_bodies(c, c->side))) break;
            if ((e = k_pre(c, c->side, 1))) break;   // step k+1, before the counter advances
            CK(c, cudaEventRecord(c->side_ev[1], c->side));
            if ((e = k_solvent(c, SOLV_COLLIDE | SOLV_STREAM | SOLV_BIN, s))) break;
            if ((e = k_rnemd(c, s, 1, 1))) break;   // before the collision of step k+1
            CK(c, cudaStreamWaitEvent(s, c->side_ev[1], 0));
            if (c->prm.sort_period >= 0 && ++c->since_sort >= c->tune.sort_period)
                if ((e = do_sort(c, 0, s, true))) break;
        }
        if ((e = k_advance(c, s))) break;
    }
    if (!e && !c->profiling) {
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(c, MPCD_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(ce));
    }
    return e;
}

int check_device_error(mpcd_ctx *c, cudaStream_t s)
{
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (h & ERR_POSITION)
        return fail(c, MPCD_ERR_STATE, "a particle or body left the periodic box in one step (|v dt| >= L)");
    if (h & ERR_INDEX) {
        int w[2] = {0, 0};
        CK(c, cudaMemcpy(w, c->d_err, sizeof w, cudaMemcpyDeviceToHost));
        return fail(c, MPCD_ERR_STATE, "an index check failed (check %d); no access was made", w[1]);
    }
    if (h & ERR_RNEMD)
        return fail(c, MPCD_ERR_STATE,
                    "momentum exchange skipped: more than %d particles in a slab or more than %d candidates "
                    "up to a slab's threshold bucket", RN_LIST, RN_CAP);
    if (h) return fail(c, MPCD_ERR_STATE, "device error word 0x%x", h);
    return MPCD_OK;
}

void clear_graphs(mpcd_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second.exec);
    c->graphs.clear();
}

}  // namespace

// ======================================================================== ABI
extern "C" {

int mpcd_create(const mpcd_params *params, int32_t n_shapes, const mpcd_shape_desc *shapes,
                int32_t n_replicas, const mpcd_replica_desc *replicas, const mpcd_allocator *allocator,
                int32_t device, mpcd_ctx **out)
{
    if (!out || !params || n_shapes < 0 || n_replicas <= 0 || !replicas || (n_shapes > 0 && !shapes))
        return MPCD_ERR_ARG;
    *out = nullptr;
    const mpcd_params &p = *params;
    if (!(p.kT > 0) || !(p.dt > 0) || !(p.m_solvent > 0) || !std::isfinite(p.alpha_deg) ||
        (p.rule != MPCD_SRD && p.rule != MPCD_AT) || (p.precision != MPCD_P32 && p.precision != MPCD_P64) ||
        (p.angular != 0 && p.angular != 1) || p.thermostat < 0 || p.thermostat > 2)
        return MPCD_ERR_ARG;
    if (allocator && (!allocator->alloc || !allocator->free)) return MPCD_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MPCD_ERR_CUDA;
    }
    mpcd_ctx *c = new mpcd_ctx();
    c->device = device;
    c->prm = p;
    if (allocator) {
        c->alloc = *allocator;
        c->use_alloc = true;
    }
    c->nrep = n_replicas;
    c->nshapes = n_shapes;
    c->realsz = p.precision == MPCD_P32 ? 4 : 8;
    c->nw = p.precision == MPCD_P32 ? (p.rule == MPCD_SRD ? Words32<0>::n : Words32<1>::n)
                                    : (p.rule == MPCD_SRD ? 6 : 8);
    c->param_bytes = p.precision == MPCD_P32 ? 32 : 64;
    if (p.sort_period > 0) c->tune.sort_period = p.sort_period;

    // shapes
    std::vector<double> tb, tm, tcent;
    for (int s = 0; s < n_shapes; ++s) {
        const mpcd_shape_desc &d = shapes[s];
        if (d.n_sites <= 0 || !d.b || !d.m || d.n_centres < 0 || (d.n_centres > 0 && !d.centres) ||
            !(d.wca_d > 1.0 || d.n_centres == 0)) {
            delete c;
            return MPCD_ERR_ARG;
        }
        DevShape S{};
        S.site_begin = (int64_t)tm.size();
        S.cent_begin = (int64_t)tcent.size() / 3;
        S.n_sites = d.n_sites;
        S.n_cent = d.n_centres;
        S.wca_d = d.wca_d;
        double M = 0, I[3] = {0, 0, 0}, com[3] = {0, 0, 0}, off = 0;
        for (int j = 0; j < d.n_sites; ++j) {
            const double *b = d.b + 3 * j;
            if (!(d.m[j] > 0) || !std::isfinite(b[0] + b[1] + b[2])) {
                delete c;
                return MPCD_ERR_ARG;
            }
            double r2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
            M += d.m[j];
            for (int k = 0; k < 3; ++k) {
                I[k] += d.m[j] * (r2 - b[k] * b[k]);
                com[k] += d.m[j] * b[k];
            }
            off = std::max({off, std::fabs(d.m[j] * b[0] * b[1]), std::fabs(d.m[j] * b[0] * b[2]),
                            std::fabs(d.m[j] * b[1] * b[2])});
            for (int k = 0; k < 3; ++k) tb.push_back(b[k]);
            tm.push_back(d.m[j]);
            // the P32 cell record counts sites and needs one site mass per context
            if (c->m_site == 0.0) c->m_site = d.m[j];
            // (so do the +a variants, whose cell sums are kept per species)
            if ((p.precision == MPCD_P32 || p.angular) && d.m[j] != c->m_site) {
                delete c;
                return MPCD_ERR_ARG;
            }
        }
        // the template must be centred and principal (Eqs. 3-5 with R = site COM)
        double Ix = 0, Iy = 0, Iz = 0;
        for (int j = 0; j < d.n_sites; ++j) {
            const double *b = d.b + 3 * j;
            Ix += d.m[j] * b[0] * b[1];
            Iy += d.m[j] * b[0] * b[2];
            Iz += d.m[j] * b[1] * b[2];
        }
        double Imax = std::max({I[0], I[1], I[2], 1e-300});
        if (std::fabs(com[0]) + std::fabs(com[1]) + std::fabs(com[2]) > 1e-8 * M * std::sqrt(Imax / M) + 1e-12 ||
            std::fabs(Ix) + std::fabs(Iy) + std::fabs(Iz) > 1e-8 * Imax) {
            delete c;
            return MPCD_ERR_ARG;
        }
        (void)off;
        S.M = M;
        for (int k = 0; k < 3; ++k) S.Ihat[k] = I[k];
        double bound = 0;
        for (int j = 0; j < d.n_centres; ++j) {
            const double *x = d.centres + 3 * j;
            bound = std::max(bound, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
            for (int k = 0; k < 3; ++k) tcent.push_back(x[k]);
        }
        S.bound = bound;
        c->max_sites = std::max(c->max_sites, d.n_sites);
        c->max_wca_d = std::max(c->max_wca_d, d.wca_d);
        c->max_cent = std::max(c->max_cent, d.n_centres);
        c->shapes.push_back(S);
    }

    // replicas, slots, cells, bodies
    std::vector<int32_t> body_shape;
    std::vector<int32_t> ids;
    int64_t slot = 0, cells = 0, bodies = 0, sites = 0, rows = 0;
    for (int r = 0; r < n_replicas; ++r) {
        const mpcd_replica_desc &d = replicas[r];
        if (d.L[0] < 3 || d.L[1] < 3 || d.L[2] < 3 || d.L[0] > 2047 || d.L[1] > 2047 || d.L[2] > 2047 ||
            d.n_solvent < 0 || d.n_bodies < 0 || (d.n_bodies > 0 && !d.body_shape) || d.stream_id < 0) {
            delete c;
            return MPCD_ERR_ARG;
        }
        ids.push_back(d.stream_id);
        DevReplica R{};
        for (int k = 0; k < 3; ++k) R.L[k] = d.L[k];
        R.cell_base = (int32_t)cells;
        R.solv_begin = slot;
        R.n_solvent = d.n_solvent;
        R.site_id_base = d.n_solvent;
        R.body_begin = bodies;
        R.body_end = bodies + d.n_bodies;
        R.site_begin = sites;
        R.row_begin = rows;
        R.key0 = (uint32_t)p.seed;
        R.key1 = (uint32_t)(p.seed >> 32) ^ (uint32_t)d.stream_id;
        for (int b = 0; b < d.n_bodies; ++b) {
            int s = d.body_shape[b];
            if (s < 0 || s >= n_shapes) {
                delete c;
                return MPCD_ERR_ARG;
            }
            body_shape.push_back(s);
            sites += c->shapes[s].n_sites;
            // forces take the minimum image of every centre pair (Eq. 1), which is
            // unique when the cutoff is below half of every box edge
            const double rcut = 0.5 * (c->shapes[s].wca_d + c->max_wca_d) - 1.0 + 1.122462048309373;
            if (d.n_bodies > 1 && (2.0 * rcut >= d.L[0] || 2.0 * rcut >= d.L[1] || 2.0 * rcut >= d.L[2])) {
                delete c;
                return MPCD_ERR_ARG;
            }
        }
        cells += (int64_t)d.L[0] * d.L[1] * d.L[2];
        slot += (d.n_solvent + 7) & ~(int64_t)7;
        bodies += d.n_bodies;
        rows += d.n_solvent;
        c->reps.push_back(R);
    }
    std::sort(ids.begin(), ids.end());
    if (cells >= ((int64_t)1 << 31) || slot >= ((int64_t)1 << 31) || sites >= ((int64_t)1 << 31) ||
        std::adjacent_find(ids.begin(), ids.end()) != ids.end()) {   // stream ids must be distinct
        delete c;
        return MPCD_ERR_ARG;
    }
    c->Ns = rows;
    c->Nslots = slot + 8;
    c->C = cells;
    c->B = bodies;
    c->Nsite = sites;

    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return MPCD_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    if (configure_body_kernels(c->max_sites, p.precision) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return MPCD_ERR_ARG;
    }

    // device memory
    auto A = [&](size_t bytes) { return dalloc(c, bytes); };
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        for (int k = 0; k < 6; ++k) ok &= (c->sol[b][k] = A(c->Nslots * c->realsz)) != nullptr;
        ok &= (c->tag[b] = (uint32_t *)A(c->Nslots * sizeof(uint32_t))) != nullptr;
    }
    ok &= (c->sums = A((size_t)c->C * c->nw * 8)) != nullptr;
    ok &= (c->params = A((size_t)c->C * c->param_bytes)) != nullptr;
    ok &= (c->d_reps = (DevReplica *)A(c->reps.size() * sizeof(DevReplica))) != nullptr;
    ok &= (c->d_shapes = (DevShape *)A(std::max<size_t>(1, c->shapes.size()) * sizeof(DevShape))) != nullptr;
    ok &= (c->d_bodies = (DevBody *)A(std::max<int64_t>(1, c->B) * sizeof(DevBody))) != nullptr;
    ok &= (c->d_bpos = (float4 *)A(std::max<int64_t>(1, c->B) * sizeof(float4))) != nullptr;
    ok &= (c->d_bpos_build = (float4 *)A(std::max<int64_t>(1, c->B) * sizeof(float4))) != nullptr;
    ok &= (c->d_nlist = (int32_t *)A(std::max<int64_t>(1, c->B) * NLIST_MAX * 4)) != nullptr;
    ok &= (c->d_ncount = (int32_t *)A(std::max<int64_t>(1, c->B) * 4)) != nullptr;
    ok &= (c->d_nl_dirty = (int *)A(8)) != nullptr;
    ok &= (c->d_pose32 = (float *)A(std::max<int64_t>(1, c->B) * POSE_W * 4)) != nullptr;
    ok &= (c->d_pose64 = (double *)A(std::max<int64_t>(1, c->B) * POSE_W * 8)) != nullptr;
    ok &= (c->d_partial = A(std::max<int64_t>(1, c->B) * SITE_WARPS * 6 * 8)) != nullptr;
    ok &= (c->d_tb = (double *)A(std::max<size_t>(1, tb.size()) * 8)) != nullptr;
    ok &= (c->d_tbf = (float *)A(std::max<size_t>(1, tb.size()) * 4)) != nullptr;
    ok &= (c->d_tm = (double *)A(std::max<size_t>(1, tm.size()) * 8)) != nullptr;
    ok &= (c->d_tmf = (float *)A(std::max<size_t>(1, tm.size()) * 4)) != nullptr;
    ok &= (c->d_tcent = (double *)A(std::max<size_t>(1, tcent.size()) * 8)) != nullptr;
    {
        int64_t nc = 0;
        for (int64_t b = 0; b < c->B; ++b) nc += c->shapes[body_shape[b]].n_cent;
        ok &= (c->d_cent64 = (double *)A((size_t)std::max<int64_t>(1, nc) * 3 * 8)) != nullptr;
        ok &= (c->d_cent32 = (float4 *)A((size_t)std::max<int64_t>(1, nc) * sizeof(float4))) != nullptr;
    }
    ok &= (c->site_v = A(std::max<int64_t>(1, c->Nsite) * 3 * c->realsz)) != nullptr;
    ok &= (c->site_cell = (int32_t *)A(std::max<int64_t>(1, c->Nsite) * 4)) != nullptr;
    ok &= (c->d_step = (int64_t *)A(8)) != nullptr;
    ok &= (c->d_err = (int *)A(8)) != nullptr;
    ok &= (c->d_tile_ctr = (int *)A(16)) != nullptr;
    ok &= (c->d_diag = (double *)A(16 * 8)) != nullptr;
    ok &= (c->counts = (int32_t *)A(c->C * 4)) != nullptr;
    ok &= (c->ex = (int32_t *)A(c->C * 4)) != nullptr;
    ok &= (c->cursor = (int32_t *)A(c->C * 4)) != nullptr;
    ok &= (c->scan_bs = (int32_t *)A(scan_block_sums_size(c->C) * 4)) != nullptr;
    ok &= (c->staging = A(std::max<int64_t>(1, c->Ns) * 6 * c->realsz)) != nullptr;
    ok &= (c->rec = A((size_t)c->Nslots * 8 * c->realsz)) != nullptr;
    ok &= (c->rs_hist = (int32_t *)A(radix_hist_ints(c->Nslots) * 4)) != nullptr;
    ok &= (c->rs_ex = (int32_t *)A(radix_hist_ints(c->Nslots) * 4)) != nullptr;
    ok &= (c->rs_bs = (int32_t *)A(scan_block_sums_size((int64_t)radix_hist_ints(c->Nslots)) * 4)) != nullptr;
    if (p.angular) {
        ok &= (c->ang_words = A((size_t)c->C * ANG_WORDS * 8)) != nullptr;
        ok &= (c->ang_params = A((size_t)c->C * angular_param_bytes(p.precision))) != nullptr;
        ok &= (c->ang_shift = (int4 *)A((size_t)c->nrep * sizeof(int4))) != nullptr;
    }
    if (!ok) {
        mpcd_destroy(c);
        return MPCD_ERR_OOM;
    }
    std::vector<float> tbf(tb.begin(), tb.end()), tmf(tm.begin(), tm.end());
    std::vector<DevBody> hb(std::max<int64_t>(1, c->B));
    {
        int64_t site = 0, cent = 0, bi = 0;
        for (int r = 0; r < n_replicas; ++r)
            for (int b = 0; b < replicas[r].n_bodies; ++b, ++bi) {
                DevBody &B = hb[bi];
                std::memset(&B, 0, sizeof B);
                B.q[0] = 1.0;
                B.shape = body_shape[bi];
                B.rep = r;
                B.site_begin = site;
                B.cent_begin = cent;
                site += c->shapes[B.shape].n_sites;
                cent += c->shapes[B.shape].n_cent;
            }
        c->n_cent_bodies = cent;
    }
    int st = MPCD_OK;
    auto H2D = [&](void *d, const void *h, size_t n) {
        if (n && cudaMemcpy(d, h, n, cudaMemcpyHostToDevice) != cudaSuccess) st = MPCD_ERR_CUDA;
    };
    H2D(c->d_reps, c->reps.data(), c->reps.size() * sizeof(DevReplica));
    H2D(c->d_shapes, c->shapes.data(), c->shapes.size() * sizeof(DevShape));
    H2D(c->d_bodies, hb.data(), c->B * sizeof(DevBody));
    H2D(c->d_tb, tb.data(), tb.size() * 8);
    H2D(c->d_tbf, tbf.data(), tbf.size() * 4);
    H2D(c->d_tm, tm.data(), tm.size() * 8);
    H2D(c->d_tmf, tmf.data(), tmf.size() * 4);
    H2D(c->d_tcent, tcent.data(), tcent.size() * 8);
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k)
            if (cudaMemset(c->sol[b][k], 0, c->Nslots * c->realsz) != cudaSuccess) st = MPCD_ERR_CUDA;
        if (cudaMemset(c->tag[b], 0xFF, c->Nslots * 4) != cudaSuccess) st = MPCD_ERR_CUDA;
    }
    if (cudaMemset(c->sums, 0, (size_t)c->C * c->nw * 8) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->params, 0, (size_t)c->C * c->param_bytes) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (c->ang_words && cudaMemset(c->ang_words, 0, (size_t)c->C * ANG_WORDS * 8) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->d_step, 0, 8) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->d_ncount, 0, std::max<int64_t>(1, c->B) * 4) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->d_bpos_build, 0, std::max<int64_t>(1, c->B) * sizeof(float4)) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->d_nl_dirty, 0xFF, sizeof(int)) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (cudaMemset(c->d_err, 0, 8) != cudaSuccess) st = MPCD_ERR_CUDA;
    // default launch form: a ring per warp of 128-particle tiles, else the
    // warp-specialised pass with the largest tile whose ring fits in shared
    // memory (the FP64 form), else direct loads
    if (staged_fits(c, 128, 3, 512)) {
        c->tune = mpcd_tuning{512, 128, 1, c->tune.sort_period, 3};
    } else {
        c->tune = mpcd_tuning{512, 2048, 1, c->tune.sort_period, 0};
        for (int t : {2048, 1536, 1024, 512})
            if (staged_fits(c, t, 2, 512)) {
                c->tune.tile = t;
                c->tune.staged = 2;
                break;
            }
    }
    build_tiles(c);
    build_ctiles(c);
    if (!st) st = upload_tiles(c);
    if (!st) {
        c->d_ctiles = (Tile *)dalloc(c, std::max<size_t>(1, c->ctiles.size()) * sizeof(Tile));
        if (!c->d_ctiles) st = MPCD_ERR_OOM;
        else H2D(c->d_ctiles, c->ctiles.data(), c->ctiles.size() * sizeof(Tile));
    }
    if (!st) {
        for (int r = 0; r < c->nrep; ++r) {
            const DevReplica &R = c->reps[r];
            for (int64_t b = R.solv_begin; b < R.solv_begin + R.n_solvent; b += 2048)
                c->io_tiles.push_back(Tile{r, 0, b, std::min<int64_t>(b + 2048, R.solv_begin + R.n_solvent)});
        }
        c->d_io_tiles = (Tile *)dalloc(c, std::max<size_t>(1, c->io_tiles.size()) * sizeof(Tile));
        if (!c->d_io_tiles) st = MPCD_ERR_OOM;
        else H2D(c->d_io_tiles, c->io_tiles.data(), c->io_tiles.size() * sizeof(Tile));
    }
    if (!st && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (!st && cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking) != cudaSuccess) st = MPCD_ERR_CUDA;
    if (!st && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) st = MPCD_ERR_CUDA;
    for (int k = 0; k <= mpcd_ctx::OUT_CHUNKS && !st; ++k)
        if (cudaEventCreateWithFlags(&c->out_ev[k], cudaEventDisableTiming) != cudaSuccess) st = MPCD_ERR_CUDA;
    for (int k = 0; k < 2 && !st; ++k) {
        if (cudaEventCreateWithFlags(&c->io_ev[k], cudaEventDisableTiming) != cudaSuccess) st = MPCD_ERR_CUDA;
        if (!st && cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming) != cudaSuccess)
            st = MPCD_ERR_CUDA;
    }
    if (st) {
        cudaGetLastError();
        mpcd_destroy(c);
        return st;
    }
    *out = c;
    return MPCD_OK;
}

int mpcd_destroy(mpcd_ctx *c)
{
    if (!c) return MPCD_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    clear_graphs(c);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->evpool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->io_stream) cudaStreamDestroy(c->io_stream);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto e : c->io_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : c->out_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : c->side_ev)
        if (e) cudaEventDestroy(e);
    for (void *p : c->allocations) {
        if (c->use_alloc) c->alloc.free(p, c->alloc.user);
        else cudaFree(p);
    }
    cudaGetLastError();
    delete c;
    return MPCD_OK;
}

int mpcd_sizes(const mpcd_ctx *c, mpcd_sizes_t *o)
{
    if (!c || !o) return MPCD_ERR_ARG;
    o->n_solvent = c->Ns;
    o->n_bodies = c->B;
    o->n_sites = c->Nsite;
    o->n_cells = c->C;
    o->n_replicas = c->nrep;
    o->n_shapes = c->nshapes;
    o->device_bytes = c->dev_bytes;
    o->sum_words = c->nw;
    o->param_bytes = c->param_bytes;
    return MPCD_OK;
}

const char *mpcd_last_error(const mpcd_ctx *c) { return c ? c->err : "null context"; }

int mpcd_set_state(mpcd_ctx *c, const mpcd_host_state *h, void *stream)
{
    CHECK_CTX(c);
    if (c->slab) return MPCD_ERR_ARG;   // a slab's particles carry box-wide ids: mpcd_slab_set_state
    if (!h || (c->Ns > 0 && (!h->x || !h->v)) || (c->B > 0 && (!h->R || !h->q || !h->P || !h->Lm)) || h->step < 0)
        return MPCD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(c, cudaSetDevice(c->device));
    // bodies: conjugate momentum p = 2 q (x) (0, Q^T L)
    std::vector<DevBody> hb(std::max<int64_t>(1, c->B));
    if (c->B) CK(c, cudaMemcpy(hb.data(), c->d_bodies, c->B * sizeof(DevBody), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < c->B; ++i) {
        DevBody &b = hb[i];
        const DevReplica &R = c->reps[b.rep];
        double nq = 0;
        for (int k = 0; k < 4; ++k) nq += h->q[4 * i + k] * h->q[4 * i + k];
        if (!(std::fabs(nq - 1.0) < 1e-6)) return MPCD_ERR_ARG;
        for (int k = 0; k < 3; ++k) {
            double x = h->R[3 * i + k];
            if (!(x >= 0.0 && x < R.L[k])) return MPCD_ERR_ARG;
            b.R[k] = x;
            b.P[k] = h->P[3 * i + k];
            b.F[k] = b.T[k] = 0.0;
            b.D[k] = 0.0;
        }
        for (int k = 0; k < 4; ++k) b.q[k] = h->q[4 * i + k];
        for (int k = 0; k < 3; ++k) b.Lm[k] = h->Lm[3 * i + k];
    }
    const size_t n3 = (size_t)c->Ns * 3;
    clear_graphs(c);
    char *stg = (char *)c->staging;
    c->cur = 0;
    StepArgs a = make_args(c);
    const StepArgs aio = make_io_args(c);
    {
        // cell-sorted storage from the tag-ordered rows: stable radix sort of
        // (cell, row) pairs in the spare buffer, then one gather (memory
        // locality only; results do not depend on the order).  The velocities
        // travel on the copy stream while the positions are keyed and sorted.
        uint32_t *kA = (uint32_t *)c->sol[1][0], *vA = (uint32_t *)c->sol[1][1];
        uint32_t *kB = (uint32_t *)c->sol[1][2], *vB = (uint32_t *)c->sol[1][3];
        if (c->Ns) {
            // positions first at full link bandwidth, then the velocities
            // while the positions are keyed and sorted
            CK(c, cudaMemcpyAsync(stg, h->x, n3 * c->realsz, cudaMemcpyHostToDevice, s));
            CK(c, cudaEventRecord(c->io_ev[0], s));
            CK(c, cudaStreamWaitEvent(c->io_stream, c->io_ev[0], 0));
            CK(c, cudaMemcpyAsync(stg + n3 * c->realsz, h->v, n3 * c->realsz, cudaMemcpyHostToDevice, c->io_stream));
            CK(c, cudaEventRecord(c->io_ev[1], c->io_stream));
        }
        launch_keys_in(aio, stg, kA, vA, c->Nslots, s);
        const int nb = key_bits((uint64_t)std::max<int64_t>(c->C - 1, 0));
        const int inB =
            launch_radix_sort(kA, vA, kB, vB, c->Nslots, nb, c->rs_hist, c->rs_ex, c->rs_bs, c->d_err, s);
        if (c->Ns) CK(c, cudaStreamWaitEvent(s, c->io_ev[1], 0));
        launch_pack_rows(aio, stg, stg + n3 * c->realsz, c->rec, c->Ns, c->num_sms, s);
        launch_gather_in(aio, c->rec, inB ? vB : vA, c->Nslots, c->Ns, c->num_sms, s);
    }
    if (c->B) CK(c, cudaMemcpyAsync(c->d_bodies, hb.data(), c->B * sizeof(DevBody), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemsetAsync(c->sums, 0, (size_t)c->C * c->nw * 8, s));
    int64_t stp = h->step;
    CK(c, cudaMemcpyAsync(c->d_step, &stp, 8, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemsetAsync(c->d_nl_dirty, 0xFF, sizeof(int), s));   // build the neighbour lists
    launch_body_force(a, 0, s);
    CK(c, cudaGetLastError());
    // the upload kernel flags positions outside [0, L): reject the state
    int flag[2] = {0, 0};
    CK(c, cudaMemcpyAsync(flag, c->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (flag[0] & ~ERR_POSITION)
        return fail(c, MPCD_ERR_STATE, "set_state: device error word 0x%x (check %d)", flag[0], flag[1]);
    if (flag[0]) {
        CK(c, cudaMemset(c->d_err, 0, sizeof(int)));
        CK(c, cudaMemset(c->tag[0], 0xFF, c->Nslots * 4));
        return MPCD_ERR_ARG;
    }
    c->step = h->step;
    c->since_sort = 0;
    c->last_key = -1;
    c->have_state = true;
    return MPCD_OK;
}

int mpcd_get_state(mpcd_ctx *c, mpcd_host_state *h, void *stream)
{
    CHECK_CTX(c);
    if (c->slab) return MPCD_ERR_ARG;   // mpcd_slab_get_state
    if (!h || (c->Ns > 0 && (!h->x || !h->v)) || (c->B > 0 && (!h->R || !h->q || !h->P || !h->Lm)))
        return MPCD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(c, cudaSetDevice(c->device));
    const size_t n3 = (size_t)c->Ns * 3;
    char *stg = (char *)c->staging;
    const StepArgs a = make_io_args(c);
    {
        // tag order from the cell-sorted storage: stable radix sort of
        // (host row, slot) pairs in the spare buffer, then a gather whose
        // stores are row-contiguous
        const int alt = c->cur ^ 1;
        uint32_t *kA = (uint32_t *)c->sol[alt][0], *vA = (uint32_t *)c->sol[alt][1];
        uint32_t *kB = (uint32_t *)c->sol[alt][2], *vB = (uint32_t *)c->sol[alt][3];
        launch_keys_out(a, kA, vA, c->Nslots, (uint32_t)c->Ns, s);
        const int nb = key_bits((uint64_t)c->Ns);
        const int inB =
            launch_radix_sort(kA, vA, kB, vB, c->Nslots, nb, c->rs_hist, c->rs_ex, c->rs_bs, c->d_err, s);
        launch_pack_slots(a, c->rec, c->Nslots, c->num_sms, s);
        // the rows leave in chunks: while chunk k travels to the host on the
        // copy stream, chunk k + 1 is gathered (one chunk for small states)
        const uint32_t *order = inB ? vB : vA;
        const int K = c->Ns >= ((int64_t)1 << 22) ? mpcd_ctx::OUT_CHUNKS : 1;
        char *sx = stg, *sv = stg + n3 * c->realsz;
        for (int k = 0; k < K && c->Ns; ++k) {
            const int64_t r0 = c->Ns * k / K, r1 = c->Ns * (k + 1) / K;
            launch_gather_rows(a, order, c->rec, sx, sv, r0, r1, c->Nslots, c->num_sms, s);
            const size_t off = (size_t)r0 * 3 * c->realsz, len = (size_t)(r1 - r0) * 3 * c->realsz;
            if (K == 1) {
                CK(c, cudaMemcpyAsync(h->x, sx, len, cudaMemcpyDeviceToHost, s));
                CK(c, cudaMemcpyAsync(h->v, sv, len, cudaMemcpyDeviceToHost, s));
                continue;
            }
            CK(c, cudaEventRecord(c->out_ev[k], s));
            CK(c, cudaStreamWaitEvent(c->io_stream, c->out_ev[k], 0));
            CK(c, cudaMemcpyAsync((char *)h->x + off, sx + off, len, cudaMemcpyDeviceToHost, c->io_stream));
            CK(c, cudaMemcpyAsync((char *)h->v + off, sv + off, len, cudaMemcpyDeviceToHost, c->io_stream));
        }
        if (K > 1) {
            CK(c, cudaEventRecord(c->out_ev[mpcd_ctx::OUT_CHUNKS], c->io_stream));
            CK(c, cudaStreamWaitEvent(s, c->out_ev[mpcd_ctx::OUT_CHUNKS], 0));
        }
    }
    CK(c, cudaGetLastError());
    std::vector<DevBody> hb(std::max<int64_t>(1, c->B));
    if (c->B) CK(c, cudaMemcpyAsync(hb.data(), c->d_bodies, c->B * sizeof(DevBody), cudaMemcpyDeviceToHost, s));
    int e = check_device_error(c, s);
    if (e) return e;
    for (int64_t i = 0; i < c->B; ++i) {
        const DevBody &b = hb[i];
        for (int k = 0; k < 3; ++k) {
            h->R[3 * i + k] = b.R[k];
            h->P[3 * i + k] = b.P[k];
            h->Lm[3 * i + k] = b.Lm[k];
        }
        for (int k = 0; k < 4; ++k) h->q[4 * i + k] = b.q[k];
    }
    h->step = c->step;
    return MPCD_OK;
}

int mpcd_stream(mpcd_ctx *c, void *stream)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    int e = k_stream(c, (cudaStream_t)stream);
    if (!e) CK(c, cudaGetLastError());
    return e;
}

int mpcd_couple(mpcd_ctx *c, int32_t phase, void *stream)
{
    CHECK_CTX(c);
    if (phase != MPCD_PRE && phase != MPCD_POST) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    int e = phase == MPCD_PRE ? k_pre(c, s) : k_post(c, s);
    if (!e && phase == MPCD_POST) e = k_vacf(c, s);
    if (!e && phase == MPCD_POST) e = k_advance(c, s);
    if (!e) CK(c, cudaGetLastError());
    return e;
}

int mpcd_collide(mpcd_ctx *c, void *stream)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    int e = k_collide(c, s);
    if (!e) CK(c, cudaGetLastError());
    c->last_key = c->step;
    return e;
}

int mpcd_step(mpcd_ctx *c, int64_t nsteps, void *stream)
{
    CHECK_CTX(c);
    if (nsteps < 0) return MPCD_ERR_ARG;
    if (nsteps == 0) return MPCD_OK;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->profiling || nsteps < 2) return run_steps(c, nsteps, s);
    auto key = std::make_tuple(nsteps, c->cur, c->since_sort);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        const int cur0 = c->cur;
        const int64_t since0 = c->since_sort, step0 = c->step, key0 = c->last_key;
        CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        int e = run_steps(c, nsteps, c->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
        if (e) {
            if (g) cudaGraphDestroy(g);
            return e;
        }
        if (ce != cudaSuccess) return fail(c, MPCD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        GraphEntry ge{};
        ce = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(c, MPCD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        ge.cur_end = c->cur;
        ge.since_end = c->since_sort;
        c->cur = cur0;
        c->since_sort = since0;
        c->step = step0;
        c->last_key = key0;
        it = c->graphs.emplace(key, ge).first;
    }
    CK(c, cudaGraphLaunch(it->second.exec, s));
    c->cur = it->second.cur_end;
    c->since_sort = it->second.since_end;
    c->last_key = c->step + nsteps - 1;
    c->step += nsteps;
    return MPCD_OK;
}

int mpcd_sort(mpcd_ctx *c, int32_t canonical, void *stream)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    int e = do_sort(c, canonical, (cudaStream_t)stream);
    if (!e) CK(c, cudaGetLastError());
    return e;
}

int mpcd_cell_order(mpcd_ctx *c, int64_t *order, int64_t *cell_start, void *stream)
{
    CHECK_CTX(c);
    if (!order || !cell_start) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = c->Ns + c->Nsite, C = c->C;
    if (!c->ord_counts) {
        c->ord_counts = (int32_t *)dalloc(c, (C + 1) * sizeof(int32_t));
        c->ord_ex = (int32_t *)dalloc(c, (C + 1) * sizeof(int32_t));
        c->ord_cursor = (int32_t *)dalloc(c, C * sizeof(int32_t));
        c->ord_bs = (int32_t *)dalloc(c, scan_block_sums_size(C + 1) * sizeof(int32_t));
        c->ord_keys = (unsigned long long *)dalloc(c, std::max<int64_t>(N, 1) * 8);
        c->ord_out = (int64_t *)dalloc(c, std::max<int64_t>(N, 1) * 8);
        c->ord_start = (int64_t *)dalloc(c, (C + 1) * 8);
        if (!c->ord_counts || !c->ord_ex || !c->ord_cursor || !c->ord_bs || !c->ord_keys || !c->ord_out ||
            !c->ord_start)
            return fail(c, MPCD_ERR_OOM, "cell-order buffers: allocation failed");
    }
    StepArgs a = make_io_args(c);
    int e = timed(c, "cell_order", (double)N * (3.0 * c->realsz + 4.0 + 4 * 8.0) + (double)C * 16.0, s, [&] {
        launch_cell_order(a, c->Ns, c->ord_counts, c->ord_ex, c->ord_cursor, c->ord_bs, c->ord_keys, c->ord_out,
                          c->ord_start, c->num_sms, s);
    });
    if (e) return e;
    CK(c, cudaGetLastError());
    if (N) CK(c, cudaMemcpyAsync(order, c->ord_out, N * 8, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(cell_start, c->ord_start, (C + 1) * 8, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return MPCD_OK;
}

// --------------------------------------------------- slab decomposition
int mpcd_create_slab(const mpcd_params *params, int32_t n_shapes, const mpcd_shape_desc *shapes, const int32_t L[3],
                     int64_t n_solvent_total, int64_t capacity, int32_t n_bodies, const int32_t *body_shape,
                     int32_t z_lo, int32_t z_hi, const mpcd_allocator *allocator, int32_t device, mpcd_ctx **out)
{
    if (!out || !params || !L || n_solvent_total < 0 || capacity < 0 || capacity > n_solvent_total ||
        n_bodies < 0 || (n_bodies > 0 && !body_shape) || params->angular != 0 || z_lo < 0 || z_hi > L[2] ||
        z_hi <= z_lo || (z_hi - z_lo < 2 && !(z_lo == 0 && z_hi == L[2])))
        return MPCD_ERR_ARG;
    mpcd_replica_desc d{};
    for (int k = 0; k < 3; ++k) d.L[k] = L[k];
    d.n_solvent = capacity;
    d.n_bodies = n_bodies;
    d.stream_id = 0;
    d.body_shape = body_shape;
    int e = mpcd_create(params, n_shapes, shapes, 1, &d, allocator, device, out);
    if (e) return e;
    mpcd_ctx *c = *out;
    c->slab = true;
    c->slab_zlo = z_lo;
    c->slab_zhi = z_hi;
    c->capacity = capacity;
    c->reps[0].site_id_base = n_solvent_total;
    const size_t nb = (size_t)std::max<int64_t>(capacity, 1);
    bool ok = true;
    for (int k = 0; k < 6 && ok; ++k) ok = (c->exp_sol[k] = dalloc(c, nb * c->realsz)) != nullptr;
    const size_t ntile = (size_t)(capacity / 2048 + 2);
    ok = ok && (c->exp_tag = (uint32_t *)dalloc(c, nb * 4)) != nullptr;
    ok = ok && (c->tag_stage = (uint32_t *)dalloc(c, nb * 4)) != nullptr;
    ok = ok && (c->slab_leave = (int32_t *)dalloc(c, ntile * 4)) != nullptr;
    ok = ok && (c->slab_leave_ex = (int32_t *)dalloc(c, ntile * 4)) != nullptr;
    ok = ok && (c->slab_bs = (int32_t *)dalloc(c, scan_block_sums_size((int64_t)ntile) * 4)) != nullptr;
    ok = ok && (c->d_dpl = (double *)dalloc(c, (size_t)std::max<int64_t>(c->B, 1) * 6 * 8)) != nullptr;
    if (!ok) {
        mpcd_destroy(c);
        *out = nullptr;
        return MPCD_ERR_OOM;
    }
    CK(c, cudaSetDevice(c->device));
    e = slab_set_count(c, 0);
    if (e) {
        mpcd_destroy(c);
        *out = nullptr;
    }
    return e;
}

int mpcd_slab_insert(mpcd_ctx *c, int64_t n, const uint32_t *tags, const void *x, const void *v, void *stream)
{
    CHECK_CTX(c);
    if (!c->slab || n < 0 || (n > 0 && (!tags || !x || !v)) || c->Ns + n > c->capacity) return MPCD_ERR_ARG;
    if (n == 0) return MPCD_OK;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    // every position inside the box (the binning rule's domain)
    const int32_t *L = c->reps[0].L;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const double xv = c->realsz == 4 ? (double)((const float *)x)[3 * i + k] : ((const double *)x)[3 * i + k];
            if (!(xv >= 0.0 && xv < (double)L[k])) return MPCD_ERR_ARG;
        }
    char *stg = (char *)c->staging;   // sized for the capacity: x and v
    const size_t n3 = (size_t)n * 3 * c->realsz;
    CK(c, cudaMemcpyAsync(stg, x, n3, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(stg + n3, v, n3, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->tag_stage, tags, n * 4, cudaMemcpyHostToDevice, s));
    StepArgs a = make_args(c);
    launch_slab_put(a, stg, stg + n3, c->tag_stage, n, c->reps[0].solv_begin + c->Ns, c->num_sms, s);
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(s));
    return slab_set_count(c, c->Ns + n);
}

int mpcd_slab_extract(mpcd_ctx *c, int64_t *n_left, void *stream)
{
    CHECK_CTX(c);
    if (!c->slab || !n_left) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    *n_left = 0;
    c->n_exp = 0;
    const int64_t nt = (int64_t)c->io_tiles.size();
    if (nt == 0) return MPCD_OK;
    StepArgs a = make_io_args(c);
    const int nxt = c->cur ^ 1;
    int e = timed(c, "slab_extract", (double)c->Ns * (6.0 * c->realsz + 4.0) * 2.0, s, [&] {
        launch_slab_count(a, c->slab_zlo, c->slab_zhi, c->slab_leave, s);
        cudaMemsetAsync(c->slab_leave + nt, 0, 4, s);
        launch_scan(c->slab_leave, c->slab_leave_ex, nt + 1, c->slab_bs, s);
        void *dst[6] = {c->sol[nxt][0], c->sol[nxt][1], c->sol[nxt][2], c->sol[nxt][3], c->sol[nxt][4], c->sol[nxt][5]};
        launch_slab_split(a, c->slab_zlo, c->slab_zhi, c->slab_leave_ex, dst, c->tag[nxt], c->exp_sol, c->exp_tag, s);
    });
    if (e) return e;
    int32_t left = 0;
    CK(c, cudaMemcpyAsync(&left, c->slab_leave_ex + nt, 4, cudaMemcpyDeviceToHost, s));
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(s));
    c->cur = nxt;
    c->n_exp = left;
    *n_left = left;
    return slab_set_count(c, c->Ns - left);
}

int mpcd_slab_export(mpcd_ctx *c, uint32_t *tags, void *x, void *v, void *stream)
{
    CHECK_CTX(c);
    if (!c->slab || (c->n_exp > 0 && (!tags || !x || !v))) return MPCD_ERR_ARG;
    if (c->n_exp == 0) return MPCD_OK;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    char *stg = (char *)c->staging;
    const size_t n3 = (size_t)c->n_exp * 3 * c->realsz;
    launch_slab_pack(c->prm.precision, c->exp_sol, c->exp_tag, c->n_exp, stg, stg + n3, c->tag_stage, c->num_sms,
                     s);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(x, stg, n3, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(v, stg + n3, n3, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(tags, c->tag_stage, c->n_exp * 4, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return MPCD_OK;
}

int mpcd_slab_set_state(mpcd_ctx *c, int64_t n, const uint32_t *tags, const void *x, const void *v, const double *R,
                        const double *q, const double *P, const double *Lm, int64_t step, void *stream)
{
    CHECK_CTX(c);
    if (!c->slab || step < 0 || (c->B > 0 && (!R || !q || !P || !Lm))) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<DevBody> hb(std::max<int64_t>(1, c->B));
    if (c->B) CK(c, cudaMemcpy(hb.data(), c->d_bodies, c->B * sizeof(DevBody), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < c->B; ++i) {
        DevBody &b = hb[i];
        double nq = 0;
        for (int k = 0; k < 4; ++k) nq += q[4 * i + k] * q[4 * i + k];
        if (!(std::fabs(nq - 1.0) < 1e-6)) return MPCD_ERR_ARG;
        for (int k = 0; k < 3; ++k) {
            if (!(R[3 * i + k] >= 0.0 && R[3 * i + k] < c->reps[0].L[k])) return MPCD_ERR_ARG;
            b.R[k] = R[3 * i + k];
            b.P[k] = P[3 * i + k];
            b.Lm[k] = Lm[3 * i + k];
            b.F[k] = b.T[k] = b.D[k] = 0.0;
        }
        for (int k = 0; k < 4; ++k) b.q[k] = q[4 * i + k];
    }
    int e = slab_set_count(c, 0);
    if (!e) e = mpcd_slab_insert(c, n, tags, x, v, stream);
    if (e) return e;
    if (c->B) CK(c, cudaMemcpyAsync(c->d_bodies, hb.data(), c->B * sizeof(DevBody), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemsetAsync(c->sums, 0, (size_t)c->C * c->nw * 8, s));
    CK(c, cudaMemcpyAsync(c->d_step, &step, 8, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemsetAsync(c->d_nl_dirty, 0xFF, sizeof(int), s));
    StepArgs a = make_args(c);
    launch_body_force(a, 0, s);
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(s));
    c->step = step;
    c->since_sort = 0;
    c->last_key = -1;
    c->have_state = true;
    return MPCD_OK;
}

int mpcd_slab_get_state(mpcd_ctx *c, int64_t *n, uint32_t *tags, void *x, void *v, double *R, double *q, double *P,
                        double *Lm, void *stream)
{
    CHECK_CTX(c);
    if (!c->slab || !n) return MPCD_ERR_ARG;
    *n = c->Ns;
    if (!tags && !x && !v && !R) return MPCD_OK;
    if ((c->Ns > 0 && (!tags || !x || !v)) || (c->B > 0 && (!R || !q || !P || !Lm))) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->Ns) {
        char *stg = (char *)c->staging;
        const size_t n3 = (size_t)c->Ns * 3 * c->realsz;
        void *cur[6] = {};
        for (int k = 0; k < 6; ++k) cur[k] = (char *)c->sol[c->cur][k] + c->reps[0].solv_begin * c->realsz;
        launch_slab_pack(c->prm.precision, cur, c->tag[c->cur] + c->reps[0].solv_begin, c->Ns, stg, stg + n3,
                         c->tag_stage, c->num_sms, s);
        CK(c, cudaGetLastError());
        CK(c, cudaMemcpyAsync(x, stg, n3, cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(v, stg + n3, n3, cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(tags, c->tag_stage, c->Ns * 4, cudaMemcpyDeviceToHost, s));
    }
    std::vector<DevBody> hb(std::max<int64_t>(1, c->B));
    if (c->B) CK(c, cudaMemcpyAsync(hb.data(), c->d_bodies, c->B * sizeof(DevBody), cudaMemcpyDeviceToHost, s));
    int e = check_device_error(c, s);
    if (e) return e;
    for (int64_t i = 0; i < c->B; ++i) {
        for (int k = 0; k < 3; ++k) {
            R[3 * i + k] = hb[i].R[k];
            P[3 * i + k] = hb[i].P[k];
            Lm[3 * i + k] = hb[i].Lm[k];
        }
        for (int k = 0; k < 4; ++k) q[4 * i + k] = hb[i].q[k];
    }
    return MPCD_OK;
}

int mpcd_collide_begin(mpcd_ctx *c, void *stream)
{
    CHECK_CTX(c);
    if (c->prm.angular) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    int e = k_solvent(c, SOLV_BIN, (cudaStream_t)stream);
    if (!e) CK(c, cudaGetLastError());
    return e;
}

int mpcd_collide_end(mpcd_ctx *c, void *stream)
{
    CHECK_CTX(c);
    if (c->prm.angular) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    int e = k_params(c, s);
    if (!e) e = k_solvent(c, SOLV_COLLIDE, s);
    if (!e) CK(c, cudaGetLastError());
    c->last_key = c->step;
    return e;
}

int mpcd_layer_words(mpcd_ctx *c, int32_t layer0, int32_t n_layers, void *words, int32_t add, void *stream)
{
    CHECK_CTX(c);
    const DevReplica &R = c->reps[0];
    if (c->nrep != 1 || !words || layer0 < 0 || n_layers <= 0 || layer0 + n_layers > R.L[2]) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t plane = (int64_t)R.L[0] * R.L[1], cell0 = (int64_t)layer0 * plane, ncell = (int64_t)n_layers * plane;
    const size_t wb = (size_t)ncell * 8;
    if (!add) {
        for (int k = 0; k < c->nw; ++k)
            CK(c, cudaMemcpyAsync((char *)words + k * wb, (char *)c->sums + ((size_t)k * c->C + cell0) * 8, wb,
                                  cudaMemcpyDeviceToHost, s));
    } else {
        if ((int64_t)(wb * c->nw) > c->words_stage_bytes) {
            c->words_stage = dalloc(c, wb * c->nw);
            if (!c->words_stage) return fail(c, MPCD_ERR_OOM, "layer words staging");
            c->words_stage_bytes = (int64_t)(wb * c->nw);
        }
        CK(c, cudaMemcpyAsync(c->words_stage, words, wb * c->nw, cudaMemcpyHostToDevice, s));
        launch_words_add(c->prm.precision, c->sums, c->nw, c->C, cell0, ncell, c->words_stage, c->num_sms, s);
        CK(c, cudaGetLastError());
    }
    CK(c, cudaStreamSynchronize(s));
    return MPCD_OK;
}

int mpcd_couple_post_partial(mpcd_ctx *c, double *dPL, void *stream)
{
    CHECK_CTX(c);
    if (!dPL || c->prm.angular) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->B == 0) return MPCD_OK;
    StepArgs a = make_args(c);
    int e = timed(c, "sites_post", (double)c->Nsite * (3.0 * c->realsz + 4.0), s,
                  [&] { launch_sites_post(a, c->max_sites, s); });
    if (e) return e;
    double *dpl = c->d_dpl;
    if (!dpl) {   // a context that is not a slab: allocated on first use
        c->d_dpl = dpl = (double *)dalloc(c, (size_t)c->B * 6 * 8);
        if (!dpl) return fail(c, MPCD_ERR_OOM, "transfer buffer");
    }
    launch_body_partial(a, dpl, s);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(dPL, dpl, (size_t)c->B * 6 * 8, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return MPCD_OK;
}

int mpcd_apply_impulse(mpcd_ctx *c, const double *dPL, void *stream)
{
    CHECK_CTX(c);
    if ((c->B > 0 && !dPL) || c->prm.angular) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->B) {
        if (!c->d_dpl) {
            c->d_dpl = (double *)dalloc(c, (size_t)c->B * 6 * 8);
            if (!c->d_dpl) return fail(c, MPCD_ERR_OOM, "transfer buffer");
        }
        CK(c, cudaMemcpyAsync(c->d_dpl, dPL, (size_t)c->B * 6 * 8, cudaMemcpyHostToDevice, s));
        StepArgs a = make_args(c);
        launch_body_apply(a, c->d_dpl, s);
    }
    int e = k_vacf(c, s);
    if (!e) e = k_advance(c, s);
    if (!e) CK(c, cudaGetLastError());
    return e;
}

int mpcd_diagnostics(mpcd_ctx *c, mpcd_diag *o, void *stream)
{
    CHECK_CTX(c);
    if (!o) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    CK(c, cudaMemsetAsync(c->d_diag, 0, 16 * 8, s));
    StepArgs a = make_io_args(c);
    launch_solvent_diag(a, c->d_diag, s);
    launch_body_diag(a, c->d_diag, s);
    CK(c, cudaGetLastError());
    double h[16];
    CK(c, cudaMemcpyAsync(h, c->d_diag, 16 * 8, cudaMemcpyDeviceToHost, s));
    int e = check_device_error(c, s);
    if (e) return e;
    const double m = c->prm.m_solvent;
    for (int k = 0; k < 3; ++k) {
        o->p_solvent[k] = m * h[k];
        o->p_bodies[k] = h[4 + k];
    }
    o->ke_solvent = 0.5 * m * h[3];
    o->ke_trans = h[7];
    o->ke_rot = h[8];
    o->step = c->step;
    return MPCD_OK;
}

int mpcd_set_body_force(mpcd_ctx *c, const double f[3], void *stream)
{
    CHECK_CTX(c);
    if (!f || !std::isfinite(f[0]) || !std::isfinite(f[1]) || !std::isfinite(f[2])) return MPCD_ERR_ARG;
    const bool on = f[0] != 0.0 || f[1] != 0.0 || f[2] != 0.0;
    if (on && (c->nrep != 1 || c->Ns == 0)) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    for (int k = 0; k < 3; ++k) c->f_ext[k] = f[k];
    clear_graphs(c);   // captured steps carry the force in their arguments
    // the stored body forces enter the next half kick: recompute them
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(c);
    if (c->have_state) launch_body_force(a, 0, s);   // else mpcd_set_state computes them
    CK(c, cudaGetLastError());
    return MPCD_OK;
}

int mpcd_body_displacements(mpcd_ctx *c, double *D, void *stream)
{
    CHECK_CTX(c);
    if (!D && c->B) return MPCD_ERR_ARG;
    if (c->B == 0) return MPCD_OK;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    // the D field of every body record: a strided copy, three doubles per body
    CK(c, cudaMemcpy2DAsync(D, 3 * sizeof(double), &c->d_bodies[0].D[0], sizeof(DevBody), 3 * sizeof(double),
                            (size_t)c->B, cudaMemcpyDeviceToHost, s));
    return check_device_error(c, s);
}

int mpcd_set_vacf(mpcd_ctx *c, int32_t n_lags, int32_t every)
{
    CHECK_CTX(c);
    if (n_lags < 0 || n_lags > MPCD_VACF_MAX_LAGS || (n_lags > 0 && every < 1)) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaDeviceSynchronize());   // no step in flight uses the buffers
    VacfArgs &g = c->vacf;
    if (n_lags > 0 && c->B > 0 && n_lags > g.n_lags) {
        // grown buffers (the old ones stay with the context until it is destroyed)
        const size_t nb = (size_t)c->B * n_lags;
        g.ring_v = (double *)dalloc(c, nb * 3 * sizeof(double));
        g.ring_w = (double *)dalloc(c, nb * 3 * sizeof(double));
        g.ct = (double *)dalloc(c, nb * sizeof(double));
        g.cr = (double *)dalloc(c, nb * sizeof(double));
        g.count = (long long *)dalloc(c, (size_t)n_lags * sizeof(long long));
        if (!g.ring_v || !g.ring_w || !g.ct || !g.cr || !g.count) return fail(c, MPCD_ERR_OOM, "vacf buffers");
    }
    if (n_lags > 0 && c->B > 0) {
        const size_t nb = (size_t)c->B * n_lags;
        CK(c, cudaMemset(g.ct, 0, nb * sizeof(double)));
        CK(c, cudaMemset(g.cr, 0, nb * sizeof(double)));
        CK(c, cudaMemset(g.count, 0, (size_t)n_lags * sizeof(long long)));
    }
    g.n_lags = n_lags;
    g.every = every;
    g.start = c->step;
    clear_graphs(c);   // captured steps include (or omit) the sampling
    return MPCD_OK;
}

int mpcd_get_vacf(mpcd_ctx *c, double *ct, double *cr, int64_t *counts, void *stream)
{
    CHECK_CTX(c);
    const VacfArgs &g = c->vacf;
    if (g.n_lags == 0) return MPCD_ERR_ARG;
    if (c->B == 0) return MPCD_OK;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)c->B * g.n_lags;
    if (ct) CK(c, cudaMemcpyAsync(ct, g.ct, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (cr) CK(c, cudaMemcpyAsync(cr, g.cr, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (counts) CK(c, cudaMemcpyAsync(counts, g.count, (size_t)g.n_lags * sizeof(long long), cudaMemcpyDeviceToHost, s));
    return check_device_error(c, s);
}

int mpcd_set_rnemd(mpcd_ctx *c, const mpcd_rnemd *cfg)
{
    CHECK_CTX(c);
    if (!cfg || cfg->reserved != 0) return MPCD_ERR_ARG;
    if (cfg->enabled) {
        const double Ly = c->nrep == 1 ? (double)c->reps[0].L[1] : 0.0;
        const mpcd_rnemd &r = *cfg;
        if (c->nrep != 1 || r.max_pairs < 0 || r.max_pairs > MPCD_RNEMD_MAX_PAIRS || r.period < 1 ||
            !(r.width > 0.0) || !(r.v_target >= 0.0) || !(r.y_a >= 0.0) || !(r.y_b >= 0.0) ||
            !(r.y_a + r.width <= Ly) || !(r.y_b + r.width <= Ly) ||
            !(r.y_a + r.width <= r.y_b || r.y_b + r.width <= r.y_a))
            return MPCD_ERR_ARG;
        CK(c, cudaSetDevice(c->device));
        if (!c->rn_hist) {
            c->rn_hist = (int32_t *)dalloc(c, 2 * RN_BUCKETS * sizeof(int32_t));
            c->rn_count = (int32_t *)dalloc(c, 2 * sizeof(int32_t));
            c->rn_list = (RnEntry *)dalloc(c, (size_t)2 * RN_LIST * sizeof(RnEntry));
            c->rn_ncand = (int32_t *)dalloc(c, 2 * sizeof(int32_t));
            c->rn_cand = (RnEntry *)dalloc(c, (size_t)2 * RN_CAP * sizeof(RnEntry));
            c->rn_tot = (double *)dalloc(c, 2 * sizeof(double));
            if (!c->rn_hist || !c->rn_count || !c->rn_list || !c->rn_ncand || !c->rn_cand || !c->rn_tot)
                return fail(c, MPCD_ERR_OOM, "exchange buffers");
        }
        CK(c, cudaDeviceSynchronize());   // no step in flight uses the buffers
        CK(c, cudaMemset(c->rn_hist, 0, 2 * RN_BUCKETS * sizeof(int32_t)));
        CK(c, cudaMemset(c->rn_count, 0, 2 * sizeof(int32_t)));
        CK(c, cudaMemset(c->rn_ncand, 0, 2 * sizeof(int32_t)));
        CK(c, cudaMemset(c->rn_tot, 0, 2 * sizeof(double)));
    }
    c->rn = *cfg;
    clear_graphs(c);   // captured steps include (or omit) the exchange
    return MPCD_OK;
}

int mpcd_rnemd_totals(mpcd_ctx *c, double *p_exchanged, int64_t *n_pairs, void *stream)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    double h[2] = {0.0, 0.0};
    if (c->rn_tot) CK(c, cudaMemcpyAsync(h, c->rn_tot, sizeof h, cudaMemcpyDeviceToHost, s));
    int e = check_device_error(c, s);
    if (e) return e;
    long long n = 0;
    memcpy(&n, &h[1], sizeof n);
    if (p_exchanged) *p_exchanged = h[0];
    if (n_pairs) *n_pairs = (int64_t)n;
    return MPCD_OK;
}

int mpcd_velocity_profile(mpcd_ctx *c, int32_t bin_axis, int32_t vel_axis, int32_t n_bins, double *mass,
                          double *momentum, void *stream)
{
    CHECK_CTX(c);
    if (bin_axis < 0 || bin_axis > 2 || vel_axis < 0 || vel_axis > 2 || n_bins < 1 ||
        n_bins > MPCD_PROFILE_MAX_BINS || !mass || !momentum)
        return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->d_profile) {
        c->d_profile = (double *)dalloc(c, 2 * MPCD_PROFILE_MAX_BINS * sizeof(double));
        if (!c->d_profile) return fail(c, MPCD_ERR_OOM, "profile buffer");
    }
    CK(c, cudaMemsetAsync(c->d_profile, 0, 2 * (size_t)n_bins * sizeof(double), s));
    StepArgs a = make_args(c);
    launch_velocity_profile(a, bin_axis, vel_axis, n_bins, c->d_profile, c->d_profile + n_bins, c->num_sms, s);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(mass, c->d_profile, (size_t)n_bins * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(momentum, c->d_profile + n_bins, (size_t)n_bins * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
    return check_device_error(c, s);
}

int mpcd_set_debug(mpcd_ctx *c, int32_t on)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    if (on && !c->dbg_sums) {
        c->dbg_sums = dalloc(c, (size_t)c->C * c->nw * 8);
        if (!c->dbg_sums) return fail(c, MPCD_ERR_OOM, "debug buffer allocation failed");
        CK(c, cudaMemset(c->dbg_sums, 0, (size_t)c->C * c->nw * 8));
    }
    c->debug = on != 0;
    clear_graphs(c);
    return MPCD_OK;
}

int mpcd_debug_cells(mpcd_ctx *c, void *sums, void *params, int32_t *site_cell, void *site_v, int32_t *shift,
                     void *stream)
{
    CHECK_CTX(c);
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (sums) {
        if (!c->dbg_sums) return MPCD_ERR_ARG;
        CK(c, cudaMemcpyAsync(sums, c->dbg_sums, (size_t)c->C * c->nw * 8, cudaMemcpyDeviceToHost, s));
    }
    if (params) CK(c, cudaMemcpyAsync(params, c->params, (size_t)c->C * c->param_bytes, cudaMemcpyDeviceToHost, s));
    if (site_cell && c->Nsite)
        CK(c, cudaMemcpyAsync(site_cell, c->site_cell, c->Nsite * 4, cudaMemcpyDeviceToHost, s));
    if (site_v && c->Nsite)
        CK(c, cudaMemcpyAsync(site_v, c->site_v, c->Nsite * 3 * c->realsz, cudaMemcpyDeviceToHost, s));
    if (shift) {
        int64_t key = c->last_key >= 0 ? c->last_key : c->step;
        for (int r = 0; r < c->nrep; ++r) grid_shift(c->reps[r], key, shift + 3 * r);
    }
    CK(c, cudaStreamSynchronize(s));
    return MPCD_OK;
}

int mpcd_set_profiling(mpcd_ctx *c, int32_t on)
{
    CHECK_CTX(c);
    c->profiling = on != 0;
    return MPCD_OK;
}

int mpcd_reset_profile(mpcd_ctx *c)
{
    CHECK_CTX(c);
    int e = drain_profile(c);
    c->prof.clear();
    return e;
}

int mpcd_get_profile(mpcd_ctx *c, mpcd_kernel_time *o, int32_t max)
{
    CHECK_CTX(c);
    int e = drain_profile(c);
    if (e) return e;
    int n = 0;
    for (auto &kv : c->prof) {
        if (o && n < max) {
            std::memset(o[n].name, 0, sizeof o[n].name);
            std::strncpy(o[n].name, kv.first.c_str(), sizeof o[n].name - 1);
            o[n].launches = kv.second.launches;
            o[n].total_ms = kv.second.ms;
            o[n].bytes_per_launch = kv.second.bytes;
        }
        ++n;
    }
    return n;
}

int mpcd_get_tuning(const mpcd_ctx *c, mpcd_tuning *o)
{
    if (!c || !o) return MPCD_ERR_ARG;
    *o = c->tune;
    return MPCD_OK;
}

int mpcd_set_tuning(mpcd_ctx *c, const mpcd_tuning *t)
{
    CHECK_CTX(c);
    if (!t) return MPCD_ERR_ARG;
    if (t->block > 0) {
        if (t->block % 32 || t->block > 512) return MPCD_ERR_ARG;
        c->tune.block = t->block;
    }
    if (t->tile > 0) {
        if (t->tile < 64) return MPCD_ERR_ARG;
        c->tune.tile = t->tile & ~7;   // tiles start on 8-element boundaries (bulk-copy alignment)
    }
    if (t->ctas_per_sm > 0) c->tune.ctas_per_sm = std::min(t->ctas_per_sm, 32);
    if (t->sort_period > 0) c->tune.sort_period = t->sort_period;
    if (t->staged >= 0) c->tune.staged = std::min(t->staged, 3);
    CK(c, cudaSetDevice(c->device));
    build_tiles(c);
    int e = upload_tiles(c);
    clear_graphs(c);
    return e;
}

int mpcd_autotune(mpcd_ctx *c, int32_t steps_per_trial, void *stream)
{
    CHECK_CTX(c);
    if (steps_per_trial <= 0) return MPCD_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    // snapshot the state (both solvent buffers are restored through `cur`)
    const size_t sb = c->Nslots * c->realsz;
    std::vector<void *> save;
    for (int k = 0; k < 6; ++k) {
        void *p = dalloc(c, sb);
        if (!p) return fail(c, MPCD_ERR_OOM, "autotune snapshot");
        CK(c, cudaMemcpyAsync(p, c->sol[c->cur][k], sb, cudaMemcpyDeviceToDevice, s));
        save.push_back(p);
    }
    void *stag = dalloc(c, c->Nslots * 4), *sbody = dalloc(c, std::max<int64_t>(1, c->B) * sizeof(DevBody));
    if (!stag || !sbody) return fail(c, MPCD_ERR_OOM, "autotune snapshot");
    CK(c, cudaMemcpyAsync(stag, c->tag[c->cur], c->Nslots * 4, cudaMemcpyDeviceToDevice, s));
    CK(c, cudaMemcpyAsync(sbody, c->d_bodies, std::max<int64_t>(1, c->B) * sizeof(DevBody), cudaMemcpyDeviceToDevice, s));
    const int64_t step0 = c->step, since0 = c->since_sort, key0 = c->last_key;
    const int cur0 = c->cur;
    // the trials must not add to the observables: the exchange totals are
    // restored after every trial, the autocorrelation sampling is paused
    double rn_tot0[2] = {0.0, 0.0};
    if (c->rn_tot) {
        CK(c, cudaMemcpyAsync(rn_tot0, c->rn_tot, sizeof rn_tot0, cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
    }
    const int32_t vacf_lags0 = c->vacf.n_lags;
    c->vacf.n_lags = 0;
    auto restore = [&]() -> int {
        if (c->rn_tot) CK(c, cudaMemcpyAsync(c->rn_tot, rn_tot0, sizeof rn_tot0, cudaMemcpyHostToDevice, s));
        c->cur = cur0;
        for (int k = 0; k < 6; ++k) CK(c, cudaMemcpyAsync(c->sol[cur0][k], save[k], sb, cudaMemcpyDeviceToDevice, s));
        CK(c, cudaMemcpyAsync(c->tag[cur0], stag, c->Nslots * 4, cudaMemcpyDeviceToDevice, s));
        CK(c, cudaMemcpyAsync(c->d_bodies, sbody, std::max<int64_t>(1, c->B) * sizeof(DevBody), cudaMemcpyDeviceToDevice, s));
        CK(c, cudaMemcpyAsync(c->d_step, &step0, 8, cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        c->step = step0;
        c->since_sort = since0;
        c->last_key = key0;
        return MPCD_OK;
    };
    mpcd_tuning best = c->tune;
    float best_ms = 1e30f;
    std::vector<mpcd_tuning> cand;
    for (int bl : {128, 256, 512})
        for (int tl : {512, 1024, 2048})
            for (int ct : {1, 2, 4, 5})
                if (staged_fits(c, tl, 1, bl) && tl >= bl) cand.push_back(mpcd_tuning{bl, tl, ct, c->tune.sort_period, 1});
    for (int bl : {256, 512})
        for (int tl : {1024, 2048})
            for (int ct : {1, 2})
                if (staged_fits(c, tl, 2, bl)) cand.push_back(mpcd_tuning{bl, tl, ct, c->tune.sort_period, 2});
    for (int bl : {256, 384, 512})
        for (int tl : {128, 256})
            for (int ct : {1, 2, 3})
                if (staged_fits(c, tl, 3, bl)) cand.push_back(mpcd_tuning{bl, tl, ct, c->tune.sort_period, 3});
    for (int bl : {256, 512})
        for (int ct : {2, 4})
            cand.push_back(mpcd_tuning{bl, 8192, ct, c->tune.sort_period, 0});
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    const bool prof = c->profiling;
    c->profiling = false;
    int st = MPCD_OK;
    // Each candidate runs the same steps from the same state twice through
    // mpcd_step, as a caller would: the first run records (and runs) its CUDA
    // graph, the second, timed, replays it.
    for (const mpcd_tuning &t : cand) {
        c->tune = t;
        build_tiles(c);
        if ((st = upload_tiles(c))) goto out;
        clear_graphs(c);
        if ((st = mpcd_step(c, steps_per_trial, s))) goto out;   // graph capture + warm-up
        if ((st = restore())) goto out;
        CK(c, cudaEventRecord(e0, s));
        if ((st = mpcd_step(c, steps_per_trial, s))) goto out;
        CK(c, cudaEventRecord(e1, s));
        CK(c, cudaEventSynchronize(e1));
        {
            float ms = 0.f;
            CK(c, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        if ((st = restore())) goto out;
    }
out:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->profiling = prof;
    c->vacf.n_lags = vacf_lags0;
    if (st) return st;
    c->tune = best;
    build_tiles(c);
    clear_graphs(c);
    return upload_tiles(c);
}

}  // extern "C"
