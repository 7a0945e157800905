/*
 * FP64 CPU oracle for one MPCD time step with rigid discrete-particle colloids
 * (arXiv 2604.14307).  TEST INFRASTRUCTURE ONLY: this file is compiled and
 * called by the test-suite, by the package's smoke check and by the benchmark's
 * CPU-baseline leg.  The product (CUDA) path never includes, links or calls it,
 * and it shares no code with that path.
 *
 * It is a plain, slow, literal restatement of the method:
 *   Sec. II.A  streaming, random grid shift, cell binning, SRD rotation,
 *              cell-level thermostat (Huang et al.), MPCD-AT rule;
 *   Sec. II.B  core-shifted WCA between colloid centres (Eq. 1);
 *              rigid body: P (Eq. 3), L (Eq. 4), rigid site velocity (Eq. 5),
 *              Miller et al. NO_SQUISH quaternion velocity Verlet;
 *   Sec. II.B.2 site thermalisation before the collision (Eq. 7), momentum
 *              transfer to the body after it and reset of the sites (Eq. 5);
 *              the naive transfer without thermalisation (negative control).
 * Floating point is FP64 throughout.  In the P32 form the stored solvent and
 * site values are float32; the oracle rounds to float exactly where that form
 * stores a value, and it takes every decision that turns floats into integers
 * (cell indices, fixed-point cell sums) on those float values, with float
 * arithmetic in the order the P32 form defines (compile with
 * -ffp-contract=off so that no multiply-add is fused).
 *
 * Readings where the paper is silent (binding on both implementations):
 *   binning  X = floor(x * 2^20), S = integer shift in [-2^19, 2^19),
 *            cell = floor((X - S) / 2^20) mod L, particles binned at x - s;
 *   RNG      Philox4x32-10 (Salmon et al., SC'11), key (seed_lo, seed_hi ^ stream id),
 *            counter (step, id, tag, j); uniform u = (x + 0.5) 2^-32;
 *            Box-Muller normals; axis z = 2u1 - 1, phi = 2 pi u2;
 *   thermostat E' ~ Gamma(3(Nc-1)/2, kT) (Eq. 6 with n = 3(Nc-1)) drawn as a sum
 *            of floor(n/2) unit exponentials plus z^2/2 for odd n (thermostat = 1),
 *            or by the rejection method of Marsaglia and Tsang (thermostat = 2);
 *            kappa = sqrt(E'/E_rel);
 *   cells with fewer than two particles are left unchanged;
 *   sort order within a cell: solvent before sites, each by ascending id;
 *   the momentum change is an impulse at the collision; centre sites are
 *   massless and do not collide;
 *   sedimentation (Sec. III.B): the body force acts at the centre of mass (the
 *   centre site of a sphere, so no torque) and is balanced by an equal share
 *   on every solvent particle of the replica;
 *   angular-momentum-conserving variants (SRD+a, MPCD-AT+a; the modification
 *   Sec. II.A cites from Noguchi and Gompper): after the rule has produced v*,
 *   every colliding cell gets the rigid rotation v' = v* + w x r_c that gives
 *   back the angular momentum about the cell's centre of mass, with
 *   Pi w = sum m r_c x (v - v*) and Pi the cell's inertia tensor about that
 *   centre (its pseudo-inverse when the members are collinear, e.g. two
 *   particles); r_c is measured on the 2^-20 lattice of the binning rule
 *   (the fractional part of (X - S) 2^-20), and the thermostat, if any, acts
 *   in the rule before the correction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the loops whose iterations are independent (one particle, one
 * cell): every output is computed by the same arithmetic in the same order as
 * with one thread, so the results do not depend on the thread count.  One
 * thread unless orc_set_threads() asks for more (and the file was compiled
 * with OpenMP). */
static int g_threads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

#define ORC_P64 0
#define ORC_P32 1
#define ORC_SRD 0
#define ORC_AT 1

enum { TAG_SHIFT = 1, TAG_AXIS = 2, TAG_THERMO = 3, TAG_THERMO_ODD = 4,
       TAG_SITE = 5, TAG_AT = 6, TAG_THERMO_MT = 7 };

typedef struct {
    double kT, dt, alpha_deg, m_solvent;
    int32_t rule, thermostat, precision, naive_transfer;
    uint64_t seed;
    int32_t n_rep;
    const int32_t *L;          /* [n_rep][3] */
    const int64_t *solv_off;   /* [n_rep+1] */
    const int64_t *body_off;   /* [n_rep+1] */
    int32_t n_shapes;
    const int64_t *site_off;   /* [n_shapes+1] */
    const double *b;           /* [sites][3] body-frame offsets */
    const double *m;           /* [sites] masses */
    const int64_t *cent_off;   /* [n_shapes+1] */
    const double *cent;        /* [centres][3] body-frame WCA centres */
    const double *wca_d;       /* [n_shapes] */
    const int32_t *body_shape; /* [bodies] */
    const int32_t *stream_id;  /* [n_rep] stream id of each replica (its index in the
                                  whole ensemble); NULL: the replica's position */
    const double *f_ext;       /* [3] constant force on every body at its centre of
                                  mass, balanced by -B f / N_s on every solvent
                                  particle of its replica (Sec. III.B
                                  sedimentation); NULL: none */
    int32_t angular;           /* 1: angular-momentum-conserving variant of the rule */
} orc_sys;

typedef struct {
    double *x, *v;      /* solvent [Ns][3] */
    double *R, *q;      /* bodies [B][3], [B][4] (w,x,y,z) */
    double *P, *Lm;     /* [B][3] linear and space-frame angular momentum */
    double *F, *T;      /* [B][3] WCA force and torque */
    int64_t step;
    double *D;          /* [B][3] unwrapped displacement (sum of the drifts); NULL: not kept */
} orc_state;

/* Optional per-collision outputs; every pointer may be NULL. */
typedef struct {
    int32_t *shift;        /* [n_rep][3] integer grid shift S */
    int32_t *cell_solvent; /* [Ns] replica-local cell index */
    int32_t *cell_site;    /* [Nsites] */
    double *site_r;        /* [Nsites][3] stored site positions */
    double *site_v;        /* [Nsites][3] velocities entering the collision */
    double *site_vpost;    /* [Nsites][3] velocities after the collision */
    int64_t *fixed;        /* [6][Ctot] fixed-point cell words (P32 form; SRD uses 4) */
    double *sums;          /* [6][Ctot]: N, M, sum m v (3), sum m v.v */
    double *cell_u;        /* [Ctot][3] */
    double *cell_axis;     /* [Ctot][3] */
    double *cell_kappa;    /* [Ctot] */
    double *cell_xibar;    /* [Ctot][3] */
    int64_t *order;        /* [Ns + Nsites] members in canonical cell order */
    int64_t *cell_start;   /* [Ctot + 1] */
    double *dP;            /* [B][3] momentum transferred to each body */
    double *dL;            /* [B][3] angular momentum transferred */
    double *cell_omega;    /* [Ctot][3] angular-momentum correction w (+a variants) */
} orc_trace;

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from its definition (Salmon, Moraes, Dror, Shaw 2011) */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(const orc_sys *s, int rep, int64_t step, uint32_t id, uint32_t tag,
                 uint32_t j, uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)step, id, tag, j };
    const uint32_t sid = s->stream_id ? (uint32_t)s->stream_id[rep] : (uint32_t)rep;
    uint32_t key[2] = { (uint32_t)s->seed, (uint32_t)(s->seed >> 32) ^ sid };
    orc_philox4x32_10(ctr, key, out);
}

static double u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

/* three standard normals from one Philox block (Box-Muller) */
static void normals3(const uint32_t w[4], double n[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = sqrt(-2.0 * log(u01(w[0])));
    double r2 = sqrt(-2.0 * log(u01(w[2])));
    n[0] = r1 * cos(two_pi * u01(w[1]));
    n[1] = r1 * sin(two_pi * u01(w[1]));
    n[2] = r2 * cos(two_pi * u01(w[3]));
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void quat_mul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* rotation matrix of a unit quaternion (w,x,y,z), body -> space */
void orc_rotation_matrix(const double q[4], double Q[3][3])
{
    double xx = q[1] * q[1], yy = q[2] * q[2], zz = q[3] * q[3];
    double xy = q[1] * q[2], xz = q[1] * q[3], yz = q[2] * q[3];
    double wx = q[0] * q[1], wy = q[0] * q[2], wz = q[0] * q[3];
    Q[0][0] = 1.0 - 2.0 * (yy + zz); Q[0][1] = 2.0 * (xy - wz);       Q[0][2] = 2.0 * (xz + wy);
    Q[1][0] = 2.0 * (xy + wz);       Q[1][1] = 1.0 - 2.0 * (xx + zz); Q[1][2] = 2.0 * (yz - wx);
    Q[2][0] = 2.0 * (xz - wy);       Q[2][1] = 2.0 * (yz + wx);       Q[2][2] = 1.0 - 2.0 * (xx + yy);
}

static void matvec(double Q[3][3], const double x[3], double o[3])
{
    for (int a = 0; a < 3; ++a) o[a] = (Q[a][0] * x[0] + Q[a][1] * x[1]) + Q[a][2] * x[2];
}

static void matTvec(double Q[3][3], const double x[3], double o[3])
{
    for (int a = 0; a < 3; ++a) o[a] = (Q[0][a] * x[0] + Q[1][a] * x[1]) + Q[2][a] * x[2];
}

/* solve the 3x3 system A x = y by Cramer's rule */
static int solve3(double A[3][3], const double y[3], double x[3])
{
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (det == 0.0) return -1;
    for (int k = 0; k < 3; ++k) {
        double B[3][3];
        memcpy(B, A, sizeof B);
        for (int a = 0; a < 3; ++a) B[a][k] = y[a];
        x[k] = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1])
              - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0])
              + B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0])) / det;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* periodic wrap and the binning rule                                  */
/* ------------------------------------------------------------------ */
static int wrap_d(double *y, double L)
{
    if (*y >= L) *y = *y - L;
    else if (*y < 0.0) { *y = *y + L; if (*y >= L) *y = 0.0; }
    return (*y >= 0.0 && *y < L) ? 0 : -1;
}

static int wrap_f(float *y, float L)
{
    if (*y >= L) *y = *y - L;
    else if (*y < 0.0f) { *y = *y + L; if (*y >= L) *y = 0.0f; }
    return (*y >= 0.0f && *y < L) ? 0 : -1;
}

/* cell index along one axis of a stored position x in [0, L) under shift S */
int32_t orc_cell_axis(double x, int32_t S, int32_t L)
{
    const int64_t D = 1048576; /* 2^20 */
    int64_t X = (int64_t)floor(x * 1048576.0);
    int64_t t = X - (int64_t)S;
    int64_t c = t / D;
    if (t % D != 0 && t < 0) c -= 1;
    c %= L;
    if (c < 0) c += L;
    return (int32_t)c;
}

static int64_t local_cell(const double r[3], const int32_t S[3], const int32_t L[3])
{
    int64_t cx = orc_cell_axis(r[0], S[0], L[0]);
    int64_t cy = orc_cell_axis(r[1], S[1], L[1]);
    int64_t cz = orc_cell_axis(r[2], S[2], L[2]);
    return cx + (int64_t)L[0] * (cy + (int64_t)L[1] * cz);
}

/* position of a stored coordinate x inside its shifted cell, in [0, 1): the
 * fractional part of (X - S) 2^-20 with X = floor(x 2^20) (the binning rule) */
static double cell_offset(double x, int32_t S)
{
    const int64_t D = 1048576; /* 2^20 */
    int64_t t = (int64_t)floor(x * 1048576.0) - (int64_t)S;
    int64_t c = t / D;
    if (t % D != 0 && t < 0) c -= 1;
    return (double)(t - c * D) * 0x1p-20;
}

/* eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
 * (Golub and Van Loan, Sec. 8.5): A = V diag(lam) V^T, columns of V */
static void sym_eig3(const double A0[3][3], double lam[3], double V[3][3])
{
    double A[3][3];
    memcpy(A, A0, sizeof A);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V[a][b] = (a == b);
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        double scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
        if (off <= 1e-300 || off <= 1e-18 * scale) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation in the (p, q) plane that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {      /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {      /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {      /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int a = 0; a < 3; ++a) lam[a] = A[a][a];
}

/* The +a correction of one cell of n members (masses m, lattice positions q
 * inside the cell, velocities v before and o after the rule): o += w x r_c
 * with w the least-norm solution of Pi w = sum m r_c x (v - o).  Eigenvalues
 * of Pi below 1e-12 of the largest count as zero (collinear members). */
static void angular_correction(int64_t n, const double *m, const double *q, const double *v, double *o,
                               double w_out[3])
{
    double M = 0, Qc[3] = { 0, 0, 0 };
    for (int64_t i = 0; i < n; ++i) {
        M += m[i];
        for (int a = 0; a < 3; ++a) Qc[a] += m[i] * q[3 * i + a];
    }
    for (int a = 0; a < 3; ++a) Qc[a] /= M;
    double Pi[3][3] = { { 0 } }, dL[3] = { 0, 0, 0 };
    for (int64_t i = 0; i < n; ++i) {
        double rc[3], dv[3], t[3];
        for (int a = 0; a < 3; ++a) { rc[a] = q[3 * i + a] - Qc[a]; dv[a] = v[3 * i + a] - o[3 * i + a]; }
        double r2 = rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi[a][b] += m[i] * ((a == b) * r2 - rc[a] * rc[b]);
        cross(rc, dv, t);
        for (int a = 0; a < 3; ++a) dL[a] += m[i] * t[a];
    }
    double lam[3], V[3][3], w[3] = { 0, 0, 0 };
    sym_eig3(Pi, lam, V);
    double lmax = fmax(fmax(lam[0], lam[1]), lam[2]);
    for (int k = 0; k < 3; ++k) {
        if (!(lam[k] > 1e-12 * lmax)) continue;
        double c = (V[0][k] * dL[0] + V[1][k] * dL[1] + V[2][k] * dL[2]) / lam[k];
        for (int a = 0; a < 3; ++a) w[a] += c * V[a][k];
    }
    for (int64_t i = 0; i < n; ++i) {
        double rc[3], t[3];
        for (int a = 0; a < 3; ++a) rc[a] = q[3 * i + a] - Qc[a];
        cross(w, rc, t);
        for (int a = 0; a < 3; ++a) o[3 * i + a] += t[a];
    }
    if (w_out) memcpy(w_out, w, sizeof w);
}

void orc_grid_shift(const orc_sys *s, int rep, int64_t step, int32_t S[3])
{
    uint32_t w[4];
    draw(s, rep, step, 0u, TAG_SHIFT, 0u, w);
    for (int a = 0; a < 3; ++a) S[a] = (int32_t)(w[a] >> 12) - (1 << 19);
}

/* ------------------------------------------------------------------ */
/* fixed-point cell record of the P32 form                              */
/* ------------------------------------------------------------------ */
/* Int64 words per cell, each an exact sum of per-particle integers:
 *   w0 = p_x + 2^48 [solvent],  w1 = p_y + 2^48 [site],  w2 = p_z
 *                                                 p = round(fl32(m v) 2^32)
 *   SRD: w3 = round(e 2^28), e = fl32(fl32(fl32(px vx) + fl32(py vy)) + fl32(pz vz))
 *   AT:  w3, w4, w5 = q                           q = round(fl32(m xi) 2^32)
 * The low 48 bits of w0 and w1 are the signed momentum sums, the high 16 bits
 * the counts of solvent particles and of sites.  The momentum quantum 2^-32 is
 * below the float32 spacing of every |m v| >= 2^-9, so the momentum words are
 * the exact sums of the stored float32 momenta (the cell momentum that the
 * collision conserves, Sec. II.A).  Rounding is to nearest, ties to even, of
 * the float value times the power of two (an exact scaling, done in double). */
#define W_COUNT ((int64_t)1 << 48)
static int64_t qs(float x, double pow2) { return (int64_t)llrint((double)x * pow2); }

static void record_terms(float m, const float v[3], int is_site, int rule, int64_t w[6])
{
    float px = m * v[0], py = m * v[1], pz = m * v[2];
    float e = (px * v[0] + py * v[1]) + pz * v[2];   /* unfused: -ffp-contract=off */
    w[0] = qs(px, 0x1p32) + (is_site ? 0 : W_COUNT);
    w[1] = qs(py, 0x1p32) + (is_site ? W_COUNT : 0);
    w[2] = qs(pz, 0x1p32);
    w[3] = rule == ORC_SRD ? qs(e, 0x1p28) : 0;
    w[4] = w[5] = 0;
}

/* a count|momentum word: signed low 48 bits and the 16-bit count above them */
static void unpack48(int64_t w, int64_t *count, int64_t *lo)
{
    int64_t l = w & (W_COUNT - 1);
    if (l >= W_COUNT / 2) l -= W_COUNT;
    *lo = l;
    *count = (int64_t)((uint64_t)(w - l) >> 48);
}

/* ------------------------------------------------------------------ */
/* rigid bodies                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double M;
    double Ihat[3];   /* body-frame principal moments (template is principal) */
} body_props;

static body_props shape_props(const orc_sys *s, int sh)
{
    body_props bp = { 0.0, { 0.0, 0.0, 0.0 } };
    for (int64_t j = s->site_off[sh]; j < s->site_off[sh + 1]; ++j) {
        const double *b = s->b + 3 * j;
        double r2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        bp.M += s->m[j];
        for (int k = 0; k < 3; ++k) bp.Ihat[k] += s->m[j] * (r2 - b[k] * b[k]);
    }
    return bp;
}

/* space-frame inertia tensor of the displaced sites, I = sum m (|d|^2 1 - d d^T) */
static void space_inertia(const orc_sys *s, int sh, double Q[3][3], double I[3][3])
{
    memset(I, 0, 9 * sizeof(double));
    for (int64_t j = s->site_off[sh]; j < s->site_off[sh + 1]; ++j) {
        double d[3];
        matvec(Q, s->b + 3 * j, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                I[a][c] += s->m[j] * ((a == c ? r2 : 0.0) - d[a] * d[c]);
    }
}

static void min_image(double d[3], const int32_t L[3])
{
    for (int a = 0; a < 3; ++a) {
        double h = 0.5 * L[a];
        if (d[a] > h) d[a] -= L[a];
        else if (d[a] < -h) d[a] += L[a];
    }
}

/* Eq. 1: core-shifted WCA energy and the magnitude of -du/dr */
void orc_wca(double r, double d, double *u, double *f)
{
    const double sigma = 1.0, eps = 1.0;
    double delta = d - sigma;
    double rcut = delta + pow(2.0, 1.0 / 6.0) * sigma;
    if (r > rcut) { *u = 0.0; *f = 0.0; return; }
    double s = sigma / (r - delta);
    double s6 = s * s * s * s * s * s;
    *u = 4.0 * eps * (s6 * s6 - s6) + eps;
    *f = 4.0 * eps * (12.0 * s6 * s6 - 6.0 * s6) / (r - delta);
}

/* WCA forces and torques on every body (pairs within a replica) */
int orc_forces(const orc_sys *s, orc_state *st, double *energy)
{
    double E = 0.0;
    for (int r = 0; r < s->n_rep; ++r) {
        const int32_t *L = s->L + 3 * r;
        for (int64_t i = s->body_off[r]; i < s->body_off[r + 1]; ++i)
            for (int a = 0; a < 3; ++a) { st->F[3 * i + a] = 0.0; st->T[3 * i + a] = 0.0; }
        for (int64_t i = s->body_off[r]; i < s->body_off[r + 1]; ++i) {
            int si = s->body_shape[i];
            double Qi[3][3];
            orc_rotation_matrix(st->q + 4 * i, Qi);
            for (int64_t j = i + 1; j < s->body_off[r + 1]; ++j) {
                int sj = s->body_shape[j];
                double Qj[3][3];
                orc_rotation_matrix(st->q + 4 * j, Qj);
                double dij = 0.5 * (s->wca_d[si] + s->wca_d[sj]);
                for (int64_t a = s->cent_off[si]; a < s->cent_off[si + 1]; ++a) {
                    double ca[3];
                    matvec(Qi, s->cent + 3 * a, ca);
                    for (int64_t c = s->cent_off[sj]; c < s->cent_off[sj + 1]; ++c) {
                        double cc[3], dv[3];
                        matvec(Qj, s->cent + 3 * c, cc);
                        for (int k = 0; k < 3; ++k)
                            dv[k] = (st->R[3 * i + k] + ca[k]) - (st->R[3 * j + k] + cc[k]);
                        min_image(dv, L);
                        double rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                        double u, fm;
                        orc_wca(rr, dij, &u, &fm);
                        if (fm == 0.0 && u == 0.0) continue;
                        E += u;
                        double f[3], ti[3], tj[3];
                        for (int k = 0; k < 3; ++k) f[k] = fm * dv[k] / rr;
                        cross(ca, f, ti);
                        cross(cc, f, tj);
                        for (int k = 0; k < 3; ++k) {
                            st->F[3 * i + k] += f[k];
                            st->F[3 * j + k] -= f[k];
                            st->T[3 * i + k] += ti[k];
                            st->T[3 * j + k] -= tj[k];
                        }
                    }
                }
            }
        }
    }
    if (energy) *energy = E;
    if (s->f_ext)   /* external force at the centre of mass: no torque */
        for (int64_t i = 0; i < s->body_off[s->n_rep]; ++i)
            for (int a = 0; a < 3; ++a) st->F[3 * i + a] += s->f_ext[a];
    return 0;
}

/* Miller et al. free-rotor sub-step about body axis k (1..3) for time h */
static void rotor(double q[4], double p[4], int k, double h, const double Ihat[3])
{
    if (Ihat[k - 1] == 0.0) return;
    double Pq[4], Pp[4];
    if (k == 1) {
        Pq[0] = -q[1]; Pq[1] = q[0]; Pq[2] = q[3]; Pq[3] = -q[2];
        Pp[0] = -p[1]; Pp[1] = p[0]; Pp[2] = p[3]; Pp[3] = -p[2];
    } else if (k == 2) {
        Pq[0] = -q[2]; Pq[1] = -q[3]; Pq[2] = q[0]; Pq[3] = q[1];
        Pp[0] = -p[2]; Pp[1] = -p[3]; Pp[2] = p[0]; Pp[3] = p[1];
    } else {
        Pq[0] = -q[3]; Pq[1] = q[2]; Pq[2] = -q[1]; Pq[3] = q[0];
        Pp[0] = -p[3]; Pp[1] = p[2]; Pp[2] = -p[1]; Pp[3] = p[0];
    }
    double zeta = (p[0] * Pq[0] + p[1] * Pq[1] + p[2] * Pq[2] + p[3] * Pq[3]) / (4.0 * Ihat[k - 1]);
    double c = cos(zeta * h), sn = sin(zeta * h);
    for (int a = 0; a < 4; ++a) {
        double nq = c * q[a] + sn * Pq[a];
        double np = c * p[a] + sn * Pp[a];
        q[a] = nq; p[a] = np;
    }
}

/* conjugate quaternion momentum p = 2 q (x) (0, L_body) from space-frame L */
static void L_to_p(const double q[4], const double Lm[3], double p[4])
{
    double Q[3][3], Lb[3];
    orc_rotation_matrix(q, Q);
    matTvec(Q, Lm, Lb);
    double v[4] = { 0.0, Lb[0], Lb[1], Lb[2] }, t[4];
    quat_mul(q, v, t);
    for (int a = 0; a < 4; ++a) p[a] = 2.0 * t[a];
}

static void p_to_L(const double q[4], const double p[4], double Lm[3])
{
    double qc[4] = { q[0], -q[1], -q[2], -q[3] }, t[4], Q[3][3];
    quat_mul(qc, p, t);
    double Lb[3] = { 0.5 * t[1], 0.5 * t[2], 0.5 * t[3] };
    orc_rotation_matrix(q, Q);
    matvec(Q, Lb, Lm);
}

/* torque kick of p over a half step h: p += 2 h q (x) (0, tau_body) */
static void torque_kick(const double q[4], double p[4], const double T[3], double h)
{
    double Q[3][3], tb[3];
    orc_rotation_matrix(q, Q);
    matTvec(Q, T, tb);
    double v[4] = { 0.0, tb[0], tb[1], tb[2] }, t[4];
    quat_mul(q, v, t);
    for (int a = 0; a < 4; ++a) p[a] += 2.0 * h * t[a];
}

/* a1 + a9: ballistic streaming of the solvent and one velocity-Verlet step
 * of the bodies (Miller NO_SQUISH rotor 3-2-1-2-3) */
int orc_stream(const orc_sys *s, orc_state *st)
{
    const double dt = s->dt;
    for (int r = 0; r < s->n_rep; ++r) {
        const int32_t *L = s->L + 3 * r;
        /* the solvent's share of the balancing force: acceleration
         * g = -B f / (N_s m); streaming v += g dt/2, x += v dt, v += g dt/2 */
        const int64_t nb = s->body_off[r + 1] - s->body_off[r], ns = s->solv_off[r + 1] - s->solv_off[r];
        double half[3] = { 0.0, 0.0, 0.0 };
        const int accel = s->f_ext && ns > 0 && (s->f_ext[0] != 0.0 || s->f_ext[1] != 0.0 || s->f_ext[2] != 0.0);
        if (accel)
            for (int a = 0; a < 3; ++a) {
                const double g = -((double)nb * s->f_ext[a]) / ((double)ns * s->m_solvent);
                half[a] = 0.5 * g * dt;
            }
        int bad = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(|| : bad)
        for (int64_t i = s->solv_off[r]; i < s->solv_off[r + 1]; ++i) {
            for (int a = 0; a < 3; ++a) {
                if (s->precision == ORC_P32) {
                    float x = (float)st->x[3 * i + a], v = (float)st->v[3 * i + a];
                    float dtf = (float)dt, h = (float)half[a];
                    if (accel) v = v + h;
                    float step = v * dtf;
                    float y = x + step;
                    if (wrap_f(&y, (float)L[a])) bad = 1;
                    if (accel) v = v + h;
                    st->x[3 * i + a] = (double)y;
                    st->v[3 * i + a] = (double)v;
                } else {
                    double v = st->v[3 * i + a];
                    if (accel) v = v + half[a];
                    double y = st->x[3 * i + a] + v * dt;
                    if (wrap_d(&y, (double)L[a])) bad = 1;
                    if (accel) v = v + half[a];
                    st->x[3 * i + a] = y;
                    st->v[3 * i + a] = v;
                }
            }
        }
        if (bad) return -1;
    }
    /* bodies: first half kick, drift, rotor */
    for (int r = 0; r < s->n_rep; ++r) {
        const int32_t *L = s->L + 3 * r;
        for (int64_t i = s->body_off[r]; i < s->body_off[r + 1]; ++i) {
            body_props bp = shape_props(s, s->body_shape[i]);
            double *q = st->q + 4 * i, p[4];
            L_to_p(q, st->Lm + 3 * i, p);
            for (int a = 0; a < 3; ++a) st->P[3 * i + a] += 0.5 * dt * st->F[3 * i + a];
            torque_kick(q, p, st->T + 3 * i, 0.5 * dt);
            for (int a = 0; a < 3; ++a) {
                const double d = dt * (st->P[3 * i + a] / bp.M);
                double y = st->R[3 * i + a] + d;
                if (wrap_d(&y, (double)L[a])) return -1;
                st->R[3 * i + a] = y;
                if (st->D) st->D[3 * i + a] += d;
            }
            rotor(q, p, 3, 0.5 * dt, bp.Ihat);
            rotor(q, p, 2, 0.5 * dt, bp.Ihat);
            rotor(q, p, 1, dt, bp.Ihat);
            rotor(q, p, 2, 0.5 * dt, bp.Ihat);
            rotor(q, p, 3, 0.5 * dt, bp.Ihat);
            double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            for (int a = 0; a < 4; ++a) q[a] /= nq;
            p_to_L(q, p, st->Lm + 3 * i);
        }
    }
    orc_forces(s, st, NULL);
    /* second half kick with the new forces */
    for (int64_t i = 0; i < s->body_off[s->n_rep]; ++i) {
        double *q = st->q + 4 * i, p[4];
        L_to_p(q, st->Lm + 3 * i, p);
        for (int a = 0; a < 3; ++a) st->P[3 * i + a] += 0.5 * dt * st->F[3 * i + a];
        torque_kick(q, p, st->T + 3 * i, 0.5 * dt);
        p_to_L(q, p, st->Lm + 3 * i);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* a2-a8: one collision at key `step`                                  */
/* ------------------------------------------------------------------ */
/* Gamma(a, 1) for a >= 1 by the squeeze-free rejection method of Marsaglia and
 * Tsang (ACM Trans. Math. Softw. 26, 363 (2000)): with d = a - 1/3 and
 * c = 1/sqrt(9 d), draw a standard normal x and a uniform u, set v = (1 + c x)^3,
 * and accept d v when v > 0 and ln u < x^2/2 + d - d v + d ln v.  Each Philox
 * block (counter word 3 = block index) gives two attempts: the Box-Muller pair
 * x = r cos(2 pi u1), r sin(2 pi u1) with r = sqrt(-2 ln u0), and the uniforms
 * of words 2 and 3.  After 64 blocks (never reached in practice: each attempt
 * is accepted with probability > 0.95) the mode-like value d is returned. */
#define MT_MAX_BLOCKS 64
static double gamma_marsaglia_tsang(const orc_sys *s, int rep, int64_t step, uint32_t cell, double a)
{
    const double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (uint32_t k = 0; k < MT_MAX_BLOCKS; ++k) {
        uint32_t w[4];
        draw(s, rep, step, cell, TAG_THERMO_MT, k, w);
        const double r = sqrt(-2.0 * log(u01(w[0])));
        const double ph = 6.283185307179586476925286766559 * u01(w[1]);
        const double xs[2] = { r * cos(ph), r * sin(ph) };
        for (int j = 0; j < 2; ++j) {
            const double x = xs[j], t = 1.0 + c * x;
            if (t <= 0.0) continue;
            const double v = t * t * t;
            if (log(u01(w[2 + j])) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
        }
    }
    return d;
}

static double thermostat_energy(const orc_sys *s, int rep, int64_t step, uint32_t cell, int64_t Nc)
{
    /* E' ~ Gamma(n/2, kT) with n = 3(Nc - 1) (Eq. 6) */
    int64_t n = 3 * (Nc - 1), nE = n / 2;
    if (s->thermostat == 2) return s->kT * gamma_marsaglia_tsang(s, rep, step, cell, 0.5 * (double)n);
    double g = 0.0;
    uint32_t w[4];
    for (int64_t i = 0; i < nE; ++i) {
        if (i % 4 == 0) draw(s, rep, step, cell, TAG_THERMO, (uint32_t)(i / 4), w);
        g += -log(u01(w[i % 4]));
    }
    if (n % 2) {
        draw(s, rep, step, cell, TAG_THERMO_ODD, 0u, w);
        double z = sqrt(-2.0 * log(u01(w[0]))) * cos(6.283185307179586476925286766559 * u01(w[1]));
        g += 0.5 * z * z;
    }
    return s->kT * g;
}

static float f32(double x) { return (float)x; }

/* SRD rotation axis of replica-local cell `cell` at collision `step`: uniform
 * on the sphere, z = 2u1 - 1, phi = 2 pi u2 (Sec. II.A) */
void orc_srd_axis(const orc_sys *s, int rep, int64_t step, uint32_t cell, double axis[3])
{
    uint32_t w[4];
    draw(s, rep, step, cell, TAG_AXIS, 0u, w);
    double z = 2.0 * u01(w[0]) - 1.0, ph = 6.283185307179586476925286766559 * u01(w[1]);
    double rho = sqrt(1.0 - z * z);
    axis[0] = rho * cos(ph); axis[1] = rho * sin(ph); axis[2] = z;
}

/* E' of the cell-level thermostat for a cell of Nc particles (Eq. 6) */
double orc_thermostat_energy(const orc_sys *s, int rep, int64_t step, uint32_t cell, int64_t Nc)
{
    return thermostat_energy(s, rep, step, cell, Nc);
}

int orc_collide(const orc_sys *s, orc_state *st, orc_trace *tr)
{
    const int p32 = (s->precision == ORC_P32);
    const double alpha = s->alpha_deg * 3.14159265358979323846264338327950288 / 180.0;
    const double ca = cos(alpha), sa = sin(alpha);
    const int64_t Ns = s->solv_off[s->n_rep];
    const int64_t B = s->body_off[s->n_rep];
    int64_t *site_base = (int64_t *)malloc((B + 1) * sizeof(int64_t));
    site_base[0] = 0;
    for (int64_t i = 0; i < B; ++i) {
        int sh = s->body_shape[i];
        site_base[i + 1] = site_base[i] + (s->site_off[sh + 1] - s->site_off[sh]);
    }
    const int64_t Nsite = site_base[B];
    int64_t *site_body = (int64_t *)malloc((Nsite + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < B; ++i)
        for (int64_t g = site_base[i]; g < site_base[i + 1]; ++g) site_body[g] = i;
    int32_t *body_rep = (int32_t *)malloc((B + 1) * sizeof(int32_t));
    for (int r = 0; r < s->n_rep; ++r)
        for (int64_t i = s->body_off[r]; i < s->body_off[r + 1]; ++i) body_rep[i] = r;
    int64_t Ctot = 0;
    int64_t *cbase = (int64_t *)malloc((s->n_rep + 1) * sizeof(int64_t));
    for (int r = 0; r < s->n_rep; ++r) {
        cbase[r] = Ctot;
        Ctot += (int64_t)s->L[3 * r] * s->L[3 * r + 1] * s->L[3 * r + 2];
    }
    cbase[s->n_rep] = Ctot;

    double *sv = (double *)malloc(3 * (Nsite ? Nsite : 1) * sizeof(double));   /* site v in */
    double *svp = (double *)malloc(3 * (Nsite ? Nsite : 1) * sizeof(double));  /* site v out */
    double *sd = (double *)malloc(3 * (Nsite ? Nsite : 1) * sizeof(double));   /* exact d_j */
    int64_t *cell_of = (int64_t *)malloc((Ns + Nsite + 1) * sizeof(int64_t)); /* global cell */
    int64_t *start = (int64_t *)calloc(Ctot + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((Ns + Nsite + 1) * sizeof(int64_t));
    double *vnew = (double *)malloc(3 * (Ns + Nsite + 1) * sizeof(double));
    double *spos = (double *)malloc(3 * (Nsite ? Nsite : 1) * sizeof(double)); /* stored site r */
    int32_t *shifts = (int32_t *)malloc(3 * (s->n_rep + 1) * sizeof(int32_t));
    int status = 0;

    for (int r = 0; r < s->n_rep; ++r) {
        const int32_t *L = s->L + 3 * r;
        int32_t S[3];
        orc_grid_shift(s, r, st->step, S);                              /* a2 */
        memcpy(shifts + 3 * r, S, sizeof S);
        if (tr && tr->shift) memcpy(tr->shift + 3 * r, S, sizeof S);
        const int64_t ns_r = s->solv_off[r + 1] - s->solv_off[r];

        /* a3 + a4: site positions from the pose, thermalisation (Eq. 7); the
         * bodies are independent */
        int berr = 0;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 4) reduction(min : berr)
        for (int64_t i = s->body_off[r]; i < s->body_off[r + 1]; ++i) {
            int sh = s->body_shape[i];
            body_props bp = shape_props(s, sh);
            double Q[3][3], I[3][3];
            orc_rotation_matrix(st->q + 4 * i, Q);
            space_inertia(s, sh, Q, I);
            double V[3], om[3];
            for (int a = 0; a < 3; ++a) V[a] = st->P[3 * i + a] / bp.M;
            if (solve3(I, st->Lm + 3 * i, om)) { berr = -2; continue; }
            double mvt[3] = { 0, 0, 0 }, Lt[3] = { 0, 0, 0 };
            int64_t nsite = s->site_off[sh + 1] - s->site_off[sh];
            double *vt = (double *)malloc(3 * nsite * sizeof(double));
            for (int64_t j = 0; j < nsite; ++j) {
                int64_t g = site_base[i] + j, tj = s->site_off[sh] + j;
                double d[3];
                matvec(Q, s->b + 3 * tj, d);
                memcpy(sd + 3 * g, d, sizeof d);
                double rr[3];
                if (p32) {
                    float Qf[3][3], bf[3];
                    for (int a = 0; a < 3; ++a) {
                        bf[a] = f32(s->b[3 * tj + a]);
                        for (int c = 0; c < 3; ++c) Qf[a][c] = f32(Q[a][c]);
                    }
                    for (int a = 0; a < 3; ++a) {
                        float t0 = Qf[a][0] * bf[0];
                        float t1 = Qf[a][1] * bf[1];
                        float t2 = Qf[a][2] * bf[2];
                        float dd = (t0 + t1) + t2;
                        float y = f32(st->R[3 * i + a]) + dd;
                        if (wrap_f(&y, (float)L[a])) { berr = -1; goto body_done; }
                        rr[a] = y;
                    }
                } else {
                    for (int a = 0; a < 3; ++a) {
                        double y = st->R[3 * i + a] + d[a];
                        if (wrap_d(&y, (double)L[a])) { berr = -1; goto body_done; }
                        rr[a] = y;
                    }
                }
                memcpy(spos + 3 * g, rr, sizeof rr);
                if (tr && tr->site_r) memcpy(tr->site_r + 3 * g, rr, sizeof rr);
                cell_of[Ns + g] = cbase[r] + local_cell(rr, S, L);
                if (!s->naive_transfer) {
                    uint32_t w[4];
                    double nn[3], mj = s->m[tj], sc = sqrt(s->kT / mj);
                    draw(s, r, st->step, (uint32_t)(ns_r + (g - site_base[s->body_off[r]])), TAG_SITE, 0u, w);
                    normals3(w, nn);
                    for (int a = 0; a < 3; ++a) vt[3 * j + a] = sc * nn[a];
                    double mv[3] = { mj * vt[3 * j], mj * vt[3 * j + 1], mj * vt[3 * j + 2] }, dx[3];
                    cross(d, mv, dx);
                    for (int a = 0; a < 3; ++a) { mvt[a] += mv[a]; Lt[a] += dx[a]; }
                }
            }
            double Vt[3] = { 0, 0, 0 }, omt[3] = { 0, 0, 0 };
            if (!s->naive_transfer) {
                for (int a = 0; a < 3; ++a) Vt[a] = mvt[a] / bp.M;
                if (solve3(I, Lt, omt)) { berr = -2; goto body_done; }
            }
            for (int64_t j = 0; j < nsite; ++j) {
                int64_t g = site_base[i] + j;
                double dom[3] = { om[0] - omt[0], om[1] - omt[1], om[2] - omt[2] }, w[3];
                cross(dom, sd + 3 * g, w);
                for (int a = 0; a < 3; ++a) {
                    double vj = V[a] - Vt[a] + w[a] + (s->naive_transfer ? 0.0 : vt[3 * j + a]);
                    sv[3 * g + a] = p32 ? (double)f32(vj) : vj;
                }
            }
        body_done:
            free(vt);
        }
        if (berr) { status = berr; goto done; }

        /* a5: bin the solvent */
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int64_t i = s->solv_off[r]; i < s->solv_off[r + 1]; ++i)
            cell_of[i] = cbase[r] + local_cell(st->x + 3 * i, S, L);
    }

    /* a5: counting sort into the canonical order (solvent, then sites) */
    if (g_threads == 1) {
        for (int64_t k = 0; k < Ns + Nsite; ++k) start[cell_of[k] + 1]++;
        for (int64_t c = 0; c < Ctot; ++c) start[c + 1] += start[c];
        int64_t *fill = (int64_t *)malloc((Ctot + 1) * sizeof(int64_t));
        memcpy(fill, start, (Ctot + 1) * sizeof(int64_t));
        for (int64_t k = 0; k < Ns + Nsite; ++k) order[fill[cell_of[k]]++] = k;
        free(fill);
    } else {
        /* the same stable sort on several threads: thread t counts and then
         * places the members of its contiguous chunk of ids, after the members
         * of the same cell from the chunks before it */
        const int T = g_threads;
        const int64_t NT = Ns + Nsite;
        int64_t *cnt = (int64_t *)calloc((size_t)T * (Ctot + 1), sizeof(int64_t));
#pragma omp parallel num_threads(T)
        {
#ifdef _OPENMP
            const int t = omp_get_thread_num();
#else
            const int t = 0;
#endif
            int64_t *my = cnt + (size_t)t * (Ctot + 1);
            for (int64_t k = NT * t / T; k < NT * (t + 1) / T; ++k) my[cell_of[k]]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t run = 0;
                for (int64_t c = 0; c < Ctot; ++c) {
                    start[c] = run;
                    for (int u = 0; u < T; ++u) {
                        const int64_t n = cnt[(size_t)u * (Ctot + 1) + c];
                        cnt[(size_t)u * (Ctot + 1) + c] = run;
                        run += n;
                    }
                }
                start[Ctot] = run;
            }
            for (int64_t k = NT * t / T; k < NT * (t + 1) / T; ++k) order[my[cell_of[k]]++] = k;
        }
        free(cnt);
    }

    /* a6 + a7: per-cell sums, collision parameters and new velocities (each
     * cell reads only its own members and writes only their new velocities) */
    for (int r = 0; r < s->n_rep; ++r) {
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1024)
        for (int64_t c = cbase[r]; c < cbase[r + 1]; ++c) {
            uint32_t lc = (uint32_t)(c - cbase[r]);
            int64_t n = start[c + 1] - start[c];
            double M = 0, pm[3] = { 0, 0, 0 }, e2 = 0;
            int64_t fx[6] = { 0, 0, 0, 0, 0, 0 };
            for (int64_t k = start[c]; k < start[c + 1]; ++k) {
                int64_t id = order[k];
                double m = id < Ns ? s->m_solvent : 0.0;
                const double *v;
                if (id < Ns) v = st->v + 3 * id;
                else {
                    int64_t g = id - Ns, b = site_body[g];
                    m = s->m[s->site_off[s->body_shape[b]] + (g - site_base[b])];
                    v = sv + 3 * g;
                }
                M += m;
                for (int a = 0; a < 3; ++a) { pm[a] += m * v[a]; e2 += m * v[a] * v[a]; }
                if (p32) {
                    float vf[3] = { f32(v[0]), f32(v[1]), f32(v[2]) };
                    int64_t w[6];
                    record_terms(f32(m), vf, id >= Ns, s->rule, w);
                    for (int q = 0; q < 6; ++q) fx[q] += w[q];
                }
            }
            double u[3] = { 0, 0, 0 };
            if (n > 0) for (int a = 0; a < 3; ++a) u[a] = pm[a] / M;
            double axis[3] = { 0, 0, 0 }, kappa = 1.0, xib[3] = { 0, 0, 0 };
            int collide = (n >= 2);
            if (s->rule == ORC_SRD && collide) {
                orc_srd_axis(s, r, st->step, lc, axis);
                if (s->thermostat && p32) {
                    /* P32 form: the kinetic energy entering the thermostat is the
                     * one its fixed-point sums carry: the exact momentum sums of
                     * the stored float32 momenta and the sum of the float32
                     * products m v.v (the same numbers as the words above),
                     * evaluated here in FP64 */
                    int64_t cnt, S1i[3];
                    unpack48(fx[0], &cnt, &S1i[0]);
                    unpack48(fx[1], &cnt, &S1i[1]);
                    S1i[2] = fx[2];
                    double S1[3] = { (double)S1i[0] * 0x1p-32, (double)S1i[1] * 0x1p-32, (double)S1i[2] * 0x1p-32 };
                    double S2 = (double)fx[3] * 0x1p-28, pp = 0.0;
                    for (int a = 0; a < 3; ++a) pp += S1[a] * S1[a];
                    double Erel = 0.5 * (S2 - pp / M);
                    double Ep = thermostat_energy(s, r, st->step, lc, n);
                    kappa = Erel > 0.0 ? sqrt(Ep / Erel) : 1.0;
                } else if (s->thermostat) {
                    double Erel = 0.0;
                    for (int64_t k = start[c]; k < start[c + 1]; ++k) {
                        int64_t id = order[k];
                        double m; const double *v;
                        if (id < Ns) { m = s->m_solvent; v = st->v + 3 * id; }
                        else {
                            int64_t g = id - Ns, b = site_body[g];
                            m = s->m[s->site_off[s->body_shape[b]] + (g - site_base[b])];
                            v = sv + 3 * g;
                        }
                        for (int a = 0; a < 3; ++a) Erel += 0.5 * m * (v[a] - u[a]) * (v[a] - u[a]);
                    }
                    double Ep = thermostat_energy(s, r, st->step, lc, n);
                    kappa = Erel > 0.0 ? sqrt(Ep / Erel) : 1.0;
                }
            }
            /* AT: xi_i ~ N(0, kT/m_i); v' = u + xi_i - sum(m xi)/M */
            double *xi = NULL;
            if (s->rule == ORC_AT && n > 0) {
                xi = (double *)malloc(3 * n * sizeof(double));
                double mx[3] = { 0, 0, 0 };
                for (int64_t k = start[c]; k < start[c + 1]; ++k) {
                    int64_t id = order[k];
                    double m; uint32_t tag;
                    if (id < Ns) { m = s->m_solvent; tag = (uint32_t)(id - s->solv_off[r]); }
                    else {
                        int64_t g = id - Ns, b = site_body[g];
                        m = s->m[s->site_off[s->body_shape[b]] + (g - site_base[b])];
                        tag = (uint32_t)((s->solv_off[r + 1] - s->solv_off[r]) + (g - site_base[s->body_off[r]]));
                    }
                    uint32_t w[4]; double nn[3];
                    draw(s, r, st->step, tag, TAG_AT, 0u, w);
                    normals3(w, nn);
                    double sc = sqrt(s->kT / m);
                    for (int a = 0; a < 3; ++a) {
                        xi[3 * (k - start[c]) + a] = sc * nn[a];
                        mx[a] += m * sc * nn[a];
                    }
                    if (p32) {
                        float q[3];
                        for (int a = 0; a < 3; ++a) q[a] = f32(m) * f32(sc * nn[a]);
                        for (int a = 0; a < 3; ++a) fx[3 + a] += qs(q[a], 0x1p32);
                    }
                }
                for (int a = 0; a < 3; ++a) xib[a] = mx[a] / M;
            }
            if (p32 && tr && tr->fixed)
                for (int q = 0; q < 6; ++q) tr->fixed[q * Ctot + c] = fx[q];
            if (tr && tr->sums) {
                tr->sums[0 * Ctot + c] = (double)n; tr->sums[1 * Ctot + c] = M;
                for (int a = 0; a < 3; ++a) tr->sums[(2 + a) * Ctot + c] = pm[a];
                tr->sums[5 * Ctot + c] = e2;
            }
            if (tr && tr->cell_u) for (int a = 0; a < 3; ++a) tr->cell_u[3 * c + a] = u[a];
            if (tr && tr->cell_axis) for (int a = 0; a < 3; ++a) tr->cell_axis[3 * c + a] = axis[a];
            if (tr && tr->cell_kappa) tr->cell_kappa[c] = kappa;
            if (tr && tr->cell_xibar) for (int a = 0; a < 3; ++a) tr->cell_xibar[3 * c + a] = xib[a];

            for (int64_t k = start[c]; k < start[c + 1]; ++k) {
                int64_t id = order[k];
                const double *v = id < Ns ? st->v + 3 * id : sv + 3 * (id - Ns);
                double *o = vnew + 3 * id;
                if (!collide) { for (int a = 0; a < 3; ++a) o[a] = v[a]; continue; }
                if (s->rule == ORC_SRD) {
                    /* Rodrigues rotation of v - u by alpha about the cell axis */
                    double w[3] = { v[0] - u[0], v[1] - u[1], v[2] - u[2] }, nx[3];
                    cross(axis, w, nx);
                    double nd = axis[0] * w[0] + axis[1] * w[1] + axis[2] * w[2];
                    for (int a = 0; a < 3; ++a)
                        o[a] = u[a] + kappa * (w[a] * ca + nx[a] * sa + axis[a] * nd * (1.0 - ca));
                } else {
                    for (int a = 0; a < 3; ++a) o[a] = u[a] + xi[3 * (k - start[c]) + a] - xib[a];
                }
            }
            free(xi);
            if (s->angular && collide) {
                /* +a: restore the cell's angular momentum about its centre of mass */
                double *mm = (double *)malloc(n * sizeof(double));
                double *qq = (double *)malloc(3 * n * sizeof(double));
                double *vv = (double *)malloc(3 * n * sizeof(double));
                double *oo = (double *)malloc(3 * n * sizeof(double));
                double w[3];
                for (int64_t k = start[c]; k < start[c + 1]; ++k) {
                    int64_t id = order[k], j = k - start[c];
                    const double *x, *v;
                    if (id < Ns) { mm[j] = s->m_solvent; x = st->x + 3 * id; v = st->v + 3 * id; }
                    else {
                        int64_t g = id - Ns, b = site_body[g];
                        mm[j] = s->m[s->site_off[s->body_shape[b]] + (g - site_base[b])];
                        x = spos + 3 * g;
                        v = sv + 3 * g;
                    }
                    for (int a = 0; a < 3; ++a) {
                        qq[3 * j + a] = cell_offset(x[a], shifts[3 * r + a]);
                        vv[3 * j + a] = v[a];
                        oo[3 * j + a] = vnew[3 * id + a];
                    }
                }
                angular_correction(n, mm, qq, vv, oo, w);
                for (int64_t k = start[c]; k < start[c + 1]; ++k)
                    for (int a = 0; a < 3; ++a) vnew[3 * order[k] + a] = oo[3 * (k - start[c]) + a];
                if (tr && tr->cell_omega) memcpy(tr->cell_omega + 3 * c, w, sizeof w);
                free(mm); free(qq); free(vv); free(oo);
            }
        }
    }

    /* solvent takes its new velocities */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < Ns; ++i)
        for (int a = 0; a < 3; ++a)
            st->v[3 * i + a] = p32 ? (double)f32(vnew[3 * i + a]) : vnew[3 * i + a];
    for (int64_t g = 0; g < Nsite; ++g)
        for (int a = 0; a < 3; ++a)
            svp[3 * g + a] = p32 ? (double)f32(vnew[3 * (Ns + g) + a]) : vnew[3 * (Ns + g) + a];

    /* a8: transfer dP, dL of the sites to their body; sites are reset (Eq. 5) */
    for (int64_t i = 0; i < B; ++i) {
        int sh = s->body_shape[i];
        double dP[3] = { 0, 0, 0 }, dL[3] = { 0, 0, 0 };
        for (int64_t j = 0; j < site_base[i + 1] - site_base[i]; ++j) {
            int64_t g = site_base[i] + j;
            double mj = s->m[s->site_off[sh] + j], dp[3], t[3];
            for (int a = 0; a < 3; ++a) dp[a] = mj * (svp[3 * g + a] - sv[3 * g + a]);
            cross(sd + 3 * g, dp, t);
            for (int a = 0; a < 3; ++a) { dP[a] += dp[a]; dL[a] += t[a]; }
        }
        for (int a = 0; a < 3; ++a) { st->P[3 * i + a] += dP[a]; st->Lm[3 * i + a] += dL[a]; }
        if (tr && tr->dP) memcpy(tr->dP + 3 * i, dP, sizeof dP);
        if (tr && tr->dL) memcpy(tr->dL + 3 * i, dL, sizeof dL);
    }

    if (tr) {
        for (int r = 0; r < s->n_rep; ++r) {
            if (tr->cell_solvent)
                for (int64_t i = s->solv_off[r]; i < s->solv_off[r + 1]; ++i)
                    tr->cell_solvent[i] = (int32_t)(cell_of[i] - cbase[r]);
        }
        for (int64_t g = 0; g < Nsite; ++g) {
            if (tr->cell_site)
                tr->cell_site[g] = (int32_t)(cell_of[Ns + g] - cbase[body_rep[site_body[g]]]);
            if (tr->site_v) memcpy(tr->site_v + 3 * g, sv + 3 * g, 3 * sizeof(double));
            if (tr->site_vpost) memcpy(tr->site_vpost + 3 * g, svp + 3 * g, 3 * sizeof(double));
        }
        if (tr->order) memcpy(tr->order, order, (Ns + Nsite) * sizeof(int64_t));
        if (tr->cell_start) memcpy(tr->cell_start, start, (Ctot + 1) * sizeof(int64_t));
    }
done:
    free(site_base); free(site_body); free(body_rep); free(cbase); free(sv); free(svp); free(sd);
    free(cell_of); free(start); free(order); free(vnew); free(spos); free(shifts);
    return status;
}

/* one full step: stream (a1, a9) then the collision (a2-a8) keyed on the
 * number of steps completed before it */
int orc_step(const orc_sys *s, orc_state *st, int64_t nsteps)
{
    for (int64_t k = 0; k < nsteps; ++k) {
        int e = orc_stream(s, st);
        if (e) return e;
        e = orc_collide(s, st, NULL);
        if (e) return e;
        st->step += 1;
    }
    return 0;
}

/* rigid site velocities of Eq. 5 for every site (used to check the reset) */
int orc_rigid_site_velocities(const orc_sys *s, const orc_state *st, double *out)
{
    int64_t g = 0;
    for (int64_t i = 0; i < s->body_off[s->n_rep]; ++i) {
        int sh = s->body_shape[i];
        body_props bp = shape_props(s, sh);
        double Q[3][3], I[3][3], om[3];
        orc_rotation_matrix(st->q + 4 * i, Q);
        space_inertia(s, sh, Q, I);
        if (solve3(I, st->Lm + 3 * i, om)) return -2;
        for (int64_t j = s->site_off[sh]; j < s->site_off[sh + 1]; ++j, ++g) {
            double d[3], w[3];
            matvec(Q, s->b + 3 * j, d);
            cross(om, d, w);
            for (int a = 0; a < 3; ++a) out[3 * g + a] = st->P[3 * i + a] / bp.M + w[a];
        }
    }
    return 0;
}

/* kinetic energies of each body: E_T = M|V|^2/2, E_R = w.I.w/2 */
int orc_body_energies(const orc_sys *s, const orc_state *st, double *ET, double *ER)
{
    for (int64_t i = 0; i < s->body_off[s->n_rep]; ++i) {
        int sh = s->body_shape[i];
        body_props bp = shape_props(s, sh);
        double Q[3][3], I[3][3], om[3];
        orc_rotation_matrix(st->q + 4 * i, Q);
        space_inertia(s, sh, Q, I);
        if (solve3(I, st->Lm + 3 * i, om)) return -2;
        const double *P = st->P + 3 * i;
        ET[i] = 0.5 * (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / bp.M;
        ER[i] = 0.5 * (om[0] * st->Lm[3 * i] + om[1] * st->Lm[3 * i + 1] + om[2] * st->Lm[3 * i + 2]);
    }
    return 0;
}

/* the three normals drawn for (replica, step, id, tag): exposed for tests */
void orc_normals(const orc_sys *s, int rep, int64_t step, uint32_t id, uint32_t tag, double out[3])
{
    uint32_t w[4];
    draw(s, rep, step, id, tag, 0u, w);
    normals3(w, out);
}
