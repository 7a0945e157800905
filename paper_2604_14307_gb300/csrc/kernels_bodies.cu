// Rigid-body and surface-site kernels (Sec. II.B and II.B.2 of arXiv 2604.14307).
//
// k_body_md     first velocity-Verlet half kick, drift of R, and the Miller et
//               al. NO_SQUISH free-rotor sequence 3-2-1-2-3 for q and its
//               conjugate momentum p = 2 q (x) (0, L_body), formed from the
//               stored space-frame L and converted back; one thread per body.
// k_body_centres the space-frame offsets Q c of every WCA centre, once per pose.
// k_body_force  core-shifted WCA (Eq. 1) between the centres of different
//               bodies of a replica, with torques, over Verlet neighbour lists
//               (FP32 bounding-sphere prefilter); one thread per body for
//               shapes of one or two centres, one warp per body otherwise;
//               the pair arithmetic in the form's precision (FP32 for P32),
//               forces and torques summed in FP64; optional second kick.
// k_vacf_sample per-body velocity autocorrelation sums (Sec. III.A).
// k_sites_pre   one CTA per body: site positions from the pose, Maxwell-
//               Boltzmann draws, per-body mean velocity and angular velocity of
//               the draws, thermalised site velocity of Eq. 7, binning of the
//               sites into the cell sums.
// k_sites_post  one CTA per body: site collision with the cell parameters,
//               segmented reduction of dP = sum m (v' - v) and
//               dL = sum d x m (v' - v) (Eqs. 3-4) into the body's momenta;
//               the sites are reset to rigid motion (Eq. 5) implicitly, since
//               the next step recomputes them from P and L.  The ANG instance
//               (angular-momentum-conserving variants) adds the cell's
//               rigid-rotation correction to the rule's velocity first.
// k_ang_sites   the sites' terms of the +a cell words: before the rule from
//               the thermalised velocities, after it from the rule's
//               velocities (recomputed with the POST coupling's arithmetic).
// This file is compiled without fused multiply-add so that the FP64 body and
// site-position arithmetic rounds the same way as the oracle.
#include "mpcd_internal.cuh"

namespace mpcd {

// a slab of a decomposed box owns the sites whose stored z lies in its range
// (bounds are integers: the comparison is exact in either precision)
template <typename Real>
__device__ __forceinline__ bool site_owned(const StepArgs &a, Real z)
{
    return !a.site_own || (z >= (Real)a.site_zlo && z < (Real)a.site_zhi);
}


// ------------------------------------------------------------- quaternions
__device__ __forceinline__ void quat_mul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// rotation matrix of a unit quaternion (w, x, y, z), body -> space
__device__ __forceinline__ void rotmat(const double q[4], double Q[9])
{
    double xx = q[1] * q[1], yy = q[2] * q[2], zz = q[3] * q[3];
    double xy = q[1] * q[2], xz = q[1] * q[3], yz = q[2] * q[3];
    double wx = q[0] * q[1], wy = q[0] * q[2], wz = q[0] * q[3];
    Q[0] = 1.0 - 2.0 * (yy + zz); Q[1] = 2.0 * (xy - wz);       Q[2] = 2.0 * (xz + wy);
    Q[3] = 2.0 * (xy + wz);       Q[4] = 1.0 - 2.0 * (xx + zz); Q[5] = 2.0 * (yz - wx);
    Q[6] = 2.0 * (xz - wy);       Q[7] = 2.0 * (yz + wx);       Q[8] = 1.0 - 2.0 * (xx + yy);
}
__device__ __forceinline__ void mv(const double Q[9], const double x[3], double o[3])
{
    for (int a = 0; a < 3; ++a) o[a] = (Q[3 * a] * x[0] + Q[3 * a + 1] * x[1]) + Q[3 * a + 2] * x[2];
}
__device__ __forceinline__ void mtv(const double Q[9], const double x[3], double o[3])
{
    for (int a = 0; a < 3; ++a) o[a] = (Q[a] * x[0] + Q[3 + a] * x[1]) + Q[6 + a] * x[2];
}

// body-frame angular momentum from p: L_body = vec(q* (x) p) / 2
__device__ __forceinline__ void body_L(const double q[4], const double p[4], double Lb[3])
{
    double qc[4] = {q[0], -q[1], -q[2], -q[3]}, t[4];
    quat_mul(qc, p, t);
    Lb[0] = 0.5 * t[1]; Lb[1] = 0.5 * t[2]; Lb[2] = 0.5 * t[3];
}
__device__ __forceinline__ void p_from_Lb(const double q[4], const double Lb[3], double p[4])
{
    double v[4] = {0.0, Lb[0], Lb[1], Lb[2]}, t[4];
    quat_mul(q, v, t);
    for (int a = 0; a < 4; ++a) p[a] = 2.0 * t[a];
}

__device__ __forceinline__ void L_to_p(const double q[4], const double Lm[3], double p[4])
{
    double Q[9], Lb[3];
    rotmat(q, Q);
    mtv(Q, Lm, Lb);
    p_from_Lb(q, Lb, p);
}
__device__ __forceinline__ void p_to_L(const double q[4], const double p[4], double Lm[3])
{
    double Q[9], Lb[3];
    body_L(q, p, Lb);
    rotmat(q, Q);
    mv(Q, Lb, Lm);
}

// p += 2 h q (x) (0, Q^T tau): torque kick over a half step h
__device__ __forceinline__ void torque_kick(const double q[4], double p[4], const double T[3], double h)
{
    double Q[9], tb[3];
    rotmat(q, Q);
    mtv(Q, T, tb);
    double v[4] = {0.0, tb[0], tb[1], tb[2]}, t[4];
    quat_mul(q, v, t);
    for (int a = 0; a < 4; ++a) p[a] += 2.0 * h * t[a];
}

// free rotation about body axis k (1..3) for time h (Miller et al. 2002)
__device__ __forceinline__ void rotor(double q[4], double p[4], int k, double h, const double Ih[3])
{
    if (Ih[k - 1] == 0.0) return;
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
    double zeta = (p[0] * Pq[0] + p[1] * Pq[1] + p[2] * Pq[2] + p[3] * Pq[3]) / (4.0 * Ih[k - 1]);
    double c = cos(zeta * h), s = sin(zeta * h);
    for (int a = 0; a < 4; ++a) {
        double nq = c * q[a] + s * Pq[a];
        double np = c * p[a] + s * Pp[a];
        q[a] = nq;
        p[a] = np;
    }
}

__device__ __forceinline__ double wrapd(double y, double L, int &bad)
{
    if (y >= L) y = y - L;
    else if (y < 0.0) { y = y + L; if (y >= L) y = 0.0; }
    bad |= !(y >= 0.0 && y < L);
    return y;
}
__device__ __forceinline__ float wrapf(float y, float L, int &bad)
{
    if (y >= L) y = y - L;
    else if (y < 0.0f) { y = y + L; if (y >= L) y = 0.0f; }
    bad |= !(y >= 0.0f && y < L);
    return y;
}

// --------------------------------------------------------------- body MD
__global__ void k_body_md(StepArgs a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    DevBody b = a.bodies[i];
    const DevShape sh = a.shapes[b.shape];
    const DevReplica r = a.reps[b.rep];
    const double dt = a.dt;
    int bad = 0;
    double p[4];
    L_to_p(b.q, b.Lm, p);
    for (int k = 0; k < 3; ++k) b.P[k] += 0.5 * dt * b.F[k];
    torque_kick(b.q, p, b.T, 0.5 * dt);
    for (int k = 0; k < 3; ++k) {
        const double d = dt * (b.P[k] / sh.M);
        b.D[k] += d;
        b.R[k] = wrapd(b.R[k] + d, (double)r.L[k], bad);
    }
    rotor(b.q, p, 3, 0.5 * dt, sh.Ihat);
    rotor(b.q, p, 2, 0.5 * dt, sh.Ihat);
    rotor(b.q, p, 1, dt, sh.Ihat);
    rotor(b.q, p, 2, 0.5 * dt, sh.Ihat);
    rotor(b.q, p, 3, 0.5 * dt, sh.Ihat);
    double nq = sqrt(b.q[0] * b.q[0] + b.q[1] * b.q[1] + b.q[2] * b.q[2] + b.q[3] * b.q[3]);
    for (int k = 0; k < 4; ++k) b.q[k] /= nq;
    p_to_L(b.q, p, b.Lm);
    DevBody *o = a.bodies + i;
    for (int k = 0; k < 3; ++k) { o->R[k] = b.R[k]; o->P[k] = b.P[k]; o->Lm[k] = b.Lm[k]; o->D[k] = b.D[k]; }
    for (int k = 0; k < 4; ++k) o->q[k] = b.q[k];
    a.bpos[i] = make_float4((float)b.R[0], (float)b.R[1], (float)b.R[2], (float)sh.bound);
    // neighbour lists stay valid while every body is within half the skin of
    // its position at the last build
    const float4 p0 = a.bpos_build[i];
    float d2 = 0.0f;
    const float Rf[3] = {(float)b.R[0], (float)b.R[1], (float)b.R[2]}, R0[3] = {p0.x, p0.y, p0.z};
    for (int k = 0; k < 3; ++k) {
        float d = Rf[k] - R0[k], h = 0.5f * r.L[k];
        d = d > h ? d - r.L[k] : (d < -h ? d + r.L[k] : d);
        d2 += d * d;
    }
    if (d2 > 0.25f * NLIST_SKIN * NLIST_SKIN) atomicOr(a.nl_dirty, 1);
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

__global__ void k_body_pos(StepArgs a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const DevBody &b = a.bodies[i];
    a.bpos[i] = make_float4((float)b.R[0], (float)b.R[1], (float)b.R[2], (float)a.shapes[b.shape].bound);
}

void launch_body_md(const StepArgs &a, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    k_body_md<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a);
}

// ------------------------------------------------------------ WCA forces
__device__ __forceinline__ void min_image(double d[3], const int32_t L[3])
{
    for (int k = 0; k < 3; ++k) {
        double h = 0.5 * L[k];
        if (d[k] > h) d[k] -= L[k];
        else if (d[k] < -h) d[k] += L[k];
    }
}

// Rotated WCA centres of every body, Q c in the space frame, once per pose (in
// FP64 and rounded to float), so that the pair loop below only adds offsets.
__global__ void k_body_centres(StepArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const DevBody &b = a.bodies[i];
    const DevShape &sh = a.shapes[b.shape];
    double Q[9];
    rotmat(b.q, Q);
    for (int c = 0; c < sh.n_cent; ++c) {
        double d[3];
        mv(Q, a.tcent + 3 * (sh.cent_begin + c), d);
        const int64_t g = b.cent_begin + c;
        for (int k = 0; k < 3; ++k) a.cent64[3 * g + k] = d[k];
        a.cent32[g] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.0f);
    }
}

template <typename Real> struct CentreOf;
template <> struct CentreOf<float> {
    __device__ static void get(const StepArgs &a, int64_t g, float c[3])
    {
        const float4 v = a.cent32[g];
        c[0] = v.x; c[1] = v.y; c[2] = v.z;
    }
};
template <> struct CentreOf<double> {
    __device__ static void get(const StepArgs &a, int64_t g, double c[3])
    {
        c[0] = a.cent64[3 * g]; c[1] = a.cent64[3 * g + 1]; c[2] = a.cent64[3 * g + 2];
    }
};

// WCA force (Eq. 1) between centre ca of body i and centre cc of body j, added
// to F and the torque c_a x f to T.  The centre-pair vector
// (R_i + c_a) - (R_j + c_c) takes its own minimum image.  Real = float for the
// P32 form (R_i - R_j formed in FP64, then the pair arithmetic in FP32), double
// for the P64 form; F and T accumulate in FP64.
template <typename Real>
__device__ __forceinline__ void centre_pair(const StepArgs &a, const DevBody &bi, const DevShape &si, int ca,
                                            const DevBody &bj, const DevShape &sj, int cc, const DevReplica &r,
                                            double F[3], double T[3])
{
    const Real rc_extra = Real(1.122462048309373);   // 2^(1/6) sigma
    const Real dij = Real(0.5 * (si.wca_d + sj.wca_d));
    const Real delta = dij - Real(1), rcut = delta + rc_extra;
    Real c_a[3], c_c[3], dv[3];
    CentreOf<Real>::get(a, bi.cent_begin + ca, c_a);
    CentreOf<Real>::get(a, bj.cent_begin + cc, c_c);
    for (int k = 0; k < 3; ++k) {
        dv[k] = (Real)(bi.R[k] - bj.R[k]) + (c_a[k] - c_c[k]);
        const Real L = (Real)r.L[k], h = Real(0.5) * L;
        if (dv[k] > h) dv[k] -= L;
        else if (dv[k] < -h) dv[k] += L;
    }
    const Real rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    if (!(rr <= rcut)) return;
    const Real sdl = Real(1) / (rr - delta);
    const Real s6 = sdl * sdl * sdl * sdl * sdl * sdl;
    const Real fm = Real(4) * (Real(12) * s6 * s6 - Real(6) * s6) / (rr - delta);
    const double f[3] = {(double)(fm * dv[0] / rr), (double)(fm * dv[1] / rr), (double)(fm * dv[2] / rr)};
    F[0] += f[0]; F[1] += f[1]; F[2] += f[2];
    T[0] += (double)c_a[1] * f[2] - (double)c_a[2] * f[1];
    T[1] += (double)c_a[2] * f[0] - (double)c_a[0] * f[2];
    T[2] += (double)c_a[0] * f[1] - (double)c_a[1] * f[0];
}

__device__ __forceinline__ bool may_interact(const StepArgs &a, const float4 &pi, const float4 &pj,
                                             const DevReplica &r, float reach)
{
    const float hx = 0.5f * r.L[0], hy = 0.5f * r.L[1], hz = 0.5f * r.L[2];
    float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
    dx = dx > hx ? dx - r.L[0] : (dx < -hx ? dx + r.L[0] : dx);
    dy = dy > hy ? dy - r.L[1] : (dy < -hy ? dy + r.L[1] : dy);
    dz = dz > hz ? dz - r.L[2] : (dz < -hz ? dz + r.L[2] : dz);
    const float lim = pi.w + pj.w + reach;
    return dx * dx + dy * dy + dz * dz <= lim * lim;
}

// candidate neighbours of each body within the bounding spheres + cutoff + skin
__global__ void k_nlist_build(StepArgs a)
{
    if (!*a.nl_dirty) return;
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= a.n_bodies) return;
    const DevBody &bi = a.bodies[i];
    const DevShape &si = a.shapes[bi.shape];
    const DevReplica r = a.reps[bi.rep];
    const float4 pi = a.bpos[i];
    const float reach = (float)(0.5 * (si.wca_d + a.max_wca_d) - 1.0 + 1.122462048309373) + NLIST_SKIN + 1e-2f;
    int count = 0;
    for (int64_t j0 = r.body_begin; j0 < r.body_end; j0 += 32) {
        const int64_t j = j0 + lane;
        bool hit = j < r.body_end && j != i && may_interact(a, pi, a.bpos[j], r, reach);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        int slot = count + __popc(m & ((1u << lane) - 1u));
        if (hit && slot < NLIST_MAX) a.nlist[(int64_t)i * NLIST_MAX + slot] = (int32_t)j;
        count += __popc(m);
    }
    if (lane == 0) {
        a.ncount[i] = count <= NLIST_MAX ? count : -1;
        a.bpos_build[i] = pi;
    }
}

// Forces done: external force, stored F and T, the second half kick (kick)
// and the pose record the site kernels read (FP64).
__device__ __forceinline__ void body_force_finish(const StepArgs &a, int64_t i, const DevBody &bi, const DevShape &si,
                                                  double F[3], const double T[3], int kick)
{
    for (int k = 0; k < 3; ++k) F[k] += a.fext[k];   // external force at the centre of mass (no torque)
    double Qi[9];
    rotmat(bi.q, Qi);
    DevBody *o = a.bodies + i;
    double P[3] = {bi.P[0], bi.P[1], bi.P[2]}, L[3] = {bi.Lm[0], bi.Lm[1], bi.Lm[2]};
    for (int k = 0; k < 3; ++k) { o->F[k] = F[k]; o->T[k] = T[k]; }
    if (kick) {
        double p[4];
        L_to_p(bi.q, L, p);
        for (int k = 0; k < 3; ++k) P[k] = bi.P[k] + 0.5 * a.dt * F[k];
        torque_kick(bi.q, p, T, 0.5 * a.dt);
        p_to_L(bi.q, p, L);
        for (int k = 0; k < 3; ++k) { o->P[k] = P[k]; o->Lm[k] = L[k]; }
    }
    // pose: Q, R, V = P/M, omega = Q Ihat^-1 Q^T L (Eq. 5)
    double V[3], Lb[3], wb[3], W[3];
    for (int k = 0; k < 3; ++k) V[k] = P[k] / si.M;
    mtv(Qi, L, Lb);
    for (int k = 0; k < 3; ++k) wb[k] = si.Ihat[k] > 0.0 ? Lb[k] / si.Ihat[k] : 0.0;
    mv(Qi, wb, W);
    double *p64 = a.pose64 + i * POSE_W;
    float *p32 = a.pose32 + i * POSE_W;
    for (int k = 0; k < 9; ++k) { p64[k] = Qi[k]; p32[k] = (float)Qi[k]; }
    for (int k = 0; k < 3; ++k) {
        p64[9 + k] = bi.R[k]; p32[9 + k] = (float)bi.R[k];
        p64[12 + k] = V[k]; p32[12 + k] = (float)V[k];
        p64[15 + k] = W[k]; p32[15 + k] = (float)W[k];
    }
    if (i == 0) *a.nl_dirty = 0;   // the lists used by this step are fresh
}

// One thread per body (shapes of one or two centres): the candidates in
// ascending order, each centre pair in turn.
template <typename Real>
__global__ void __launch_bounds__(128) k_body_force(StepArgs a, int kick)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const DevBody bi = a.bodies[i];
    const DevShape si = a.shapes[bi.shape];
    const DevReplica r = a.reps[bi.rep];
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    const int n = a.ncount[i];
    if (n >= 0 && n <= NLIST_MAX) {
        for (int e = 0; e < n; ++e) {
            const int64_t j = a.nlist[i * NLIST_MAX + e];
            if (j < r.body_begin || j >= r.body_end) continue;
            const DevBody &bj = a.bodies[j];
            const DevShape &sj = a.shapes[bj.shape];
            for (int ca = 0; ca < si.n_cent; ++ca)
                for (int cc = 0; cc < sj.n_cent; ++cc) centre_pair<Real>(a, bi, si, ca, bj, sj, cc, r, F, T);
        }
    } else {
        const float4 pi = a.bpos[i];
        const float reach = (float)(0.5 * (si.wca_d + a.max_wca_d) - 1.0 + 1.122462048309373) + 1e-2f;
        for (int64_t j = r.body_begin; j < r.body_end; ++j) {
            if (j == i || !may_interact(a, pi, a.bpos[j], r, reach)) continue;
            const DevBody &bj = a.bodies[j];
            const DevShape &sj = a.shapes[bj.shape];
            for (int ca = 0; ca < si.n_cent; ++ca)
                for (int cc = 0; cc < sj.n_cent; ++cc) centre_pair<Real>(a, bi, si, ca, bj, sj, cc, r, F, T);
        }
    }
    body_force_finish(a, i, bi, si, F, T, kick);
}

// One warp per body (shapes with many centres, e.g. rods): the lanes take the
// (neighbour, centre, centre) triples of the body's candidates in turn, each
// lane summing its triples in order, and a fixed shuffle tree adds the lanes,
// so the result depends only on the candidate list.
template <typename Real>
__global__ void __launch_bounds__(128) k_body_force_warp(StepArgs a, int kick)
{
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= a.n_bodies) return;   // uniform over the warp
    const DevBody bi = a.bodies[i];
    const DevShape si = a.shapes[bi.shape];
    const DevReplica r = a.reps[bi.rep];
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    const int n = a.ncount[i];
    const int nci = si.n_cent, maxc = max(a.max_cent, 1);
    if (n >= 0 && n <= NLIST_MAX) {
        const int per = nci * maxc;
        for (int t = lane; t < n * per; t += 32) {
            const int e = t / per, rem = t - e * per, ca = rem / maxc, cc = rem - ca * maxc;
            const int64_t j = a.nlist[i * NLIST_MAX + e];
            if (j < r.body_begin || j >= r.body_end) continue;
            const DevBody &bj = a.bodies[j];
            const DevShape &sj = a.shapes[bj.shape];
            if (cc < sj.n_cent) centre_pair<Real>(a, bi, si, ca, bj, sj, cc, r, F, T);
        }
    } else {
        // the list overflowed: every body of the replica, prefiltered
        const float4 pi = a.bpos[i];
        const float reach = (float)(0.5 * (si.wca_d + a.max_wca_d) - 1.0 + 1.122462048309373) + 1e-2f;
        for (int64_t j = r.body_begin + lane; j < r.body_end; j += 32) {
            if (j == i || !may_interact(a, pi, a.bpos[j], r, reach)) continue;
            const DevBody &bj = a.bodies[j];
            const DevShape &sj = a.shapes[bj.shape];
            for (int ca = 0; ca < nci; ++ca)
                for (int cc = 0; cc < sj.n_cent; ++cc) centre_pair<Real>(a, bi, si, ca, bj, sj, cc, r, F, T);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F[k] += __shfl_down_sync(0xffffffffu, F[k], o);
            T[k] += __shfl_down_sync(0xffffffffu, T[k], o);
        }
    if (lane == 0) body_force_finish(a, i, bi, si, F, T, kick);
}

void launch_body_force(const StepArgs &a, int kick, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    if (!kick) k_body_pos<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a);
    k_body_centres<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a);
    const int wpb = 4;
    k_nlist_build<<<(a.n_bodies + wpb - 1) / wpb, 32 * wpb, 0, s>>>(a);
    if (a.max_cent <= 2) {   // spheres, dumbbells: one thread per body
        const unsigned grid = (unsigned)((a.n_bodies + 127) / 128);
        if (a.precision == 1) k_body_force<float><<<grid, 128, 0, s>>>(a, kick);
        else k_body_force<double><<<grid, 128, 0, s>>>(a, kick);
    } else {                 // many centres: one warp per body
        const unsigned grid = (unsigned)((a.n_bodies + wpb - 1) / wpb);
        if (a.precision == 1) k_body_force_warp<float><<<grid, 32 * wpb, 0, s>>>(a, kick);
        else k_body_force_warp<double><<<grid, 32 * wpb, 0, s>>>(a, kick);
    }
}

// ---------------------------------------------------------------- sites
// (x + 1/2) 2^-32 from all 32 bits, relative error <= 2^-24 (never 0; 1 only
// when x rounds up to 2^32)
__device__ __forceinline__ float u01f(uint32_t x)
{
    return __fmaf_rn(__uint2float_rn(x), 2.3283064365386962890625e-10f, 1.16415321826934814453125e-10f);
}
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386962890625e-10; }
// -2 ln u, accurate near u = 1 through the exact complement 1 - u
__device__ __forceinline__ float neg2log(uint32_t x)
{
    return (x & 0x80000000u) ? -2.0f * log1pf(-u01f(~x)) : -2.0f * __logf(u01f(x));
}
// Box-Muller; the angles are shifted by pi into [-pi, pi) where the fast
// sine/cosine are accurate: cos(2 pi u) = -cos(2 pi (u - 1/2))
__device__ __forceinline__ void normals3(uint4 w, float n[3])
{
    const float r1 = sqrtf(neg2log(w.x)), r2 = sqrtf(neg2log(w.z));
    float s1, c1;
    __sincosf(6.283185307179586f * (u01f(w.y) - 0.5f), &s1, &c1);
    n[0] = -r1 * c1; n[1] = -r1 * s1;
    n[2] = -r2 * __cosf(6.283185307179586f * (u01f(w.w) - 0.5f));
}
__device__ __forceinline__ void normals3(uint4 w, double n[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = sqrt(-2.0 * log(u01d(w.x))), r2 = sqrt(-2.0 * log(u01d(w.z)));
    double s1, c1;
    sincos(two_pi * u01d(w.y), &s1, &c1);
    n[0] = r1 * c1; n[1] = r1 * s1; n[2] = r2 * cos(two_pi * u01d(w.w));
}
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

// Site geometry of the two forms.  P32: d = Qf bf in float (three products,
// two adds), r = fl32(R) + d; P64: d = Q b in double.  Both wrapped into [0, L).
template <typename Real> struct Pose {
    Real Q[9], R[3], V[3], W[3];
};
__device__ __forceinline__ void site_geom(const StepArgs &a, int64_t t, const Pose<float> &P, const DevReplica &r,
                                          float d[3], float x[3], int &bad)
{
    const float *b = a.tbf + 3 * t;
    for (int k = 0; k < 3; ++k) {
        const float t0 = __fmul_rn(P.Q[3 * k], b[0]);
        const float t1 = __fmul_rn(P.Q[3 * k + 1], b[1]);
        const float t2 = __fmul_rn(P.Q[3 * k + 2], b[2]);
        d[k] = __fadd_rn(__fadd_rn(t0, t1), t2);
        x[k] = wrapf(__fadd_rn(P.R[k], d[k]), (float)r.L[k], bad);
    }
}
__device__ __forceinline__ void site_geom(const StepArgs &a, int64_t t, const Pose<double> &P, const DevReplica &r,
                                          double d[3], double x[3], int &bad)
{
    mv(P.Q, a.tb + 3 * t, d);
    for (int k = 0; k < 3; ++k) x[k] = wrapd(P.R[k] + d[k], (double)r.L[k], bad);
}
__device__ __forceinline__ const float *pose_ptr(const StepArgs &a, int b, float) { return a.pose32 + (int64_t)b * POSE_W; }
__device__ __forceinline__ const double *pose_ptr(const StepArgs &a, int b, double) { return a.pose64 + (int64_t)b * POSE_W; }

template <typename Real> __device__ __forceinline__ Real site_mass(const StepArgs &a, int64_t t);
template <> __device__ __forceinline__ float site_mass<float>(const StepArgs &a, int64_t t) { return a.tmf[t]; }
template <> __device__ __forceinline__ double site_mass<double>(const StepArgs &a, int64_t t) { return a.tm[t]; }

// sum six per-thread values over the CTA in the form's precision (thread 0 gets it)
template <typename Real>
__device__ void block_sum6(Real (&v)[6], Real (*scratch)[6], Real *out)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < 6; ++k) scratch[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) {
            Real s = 0;
            for (int w = 0; w < SITE_WARPS; ++w) s += scratch[w][k];
            out[k] = s;
        }
    __syncthreads();
}

// FP64 form: the sites' contributions to the double sum arrays
__device__ __forceinline__ void add_sums64(const StepArgs &a, int64_t c, double m, const double v[3],
                                           const double xi[3])
{
    double *S = reinterpret_cast<double *>(a.sums);
    const int64_t C = a.n_cells;
    atomicAdd(S + c, 1.0);
    atomicAdd(S + C + c, m);
    for (int k = 0; k < 3; ++k) atomicAdd(S + (2 + k) * C + c, m * v[k]);
    if (a.rule == 0) atomicAdd(S + 5 * C + c, m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    else for (int k = 0; k < 3; ++k) atomicAdd(S + (5 + k) * C + c, m * xi[k]);
}

template <typename Real> __device__ __forceinline__ void load_cell(const StepArgs &a, int64_t c, Real p[8]);
template <> __device__ __forceinline__ void load_cell<float>(const StepArgs &a, int64_t c, float p[8])
{
    const float4 *r = reinterpret_cast<const float4 *>(a.params) + 2 * c;
    float4 x = r[0], y = r[1];
    p[0] = x.x; p[1] = x.y; p[2] = x.z; p[3] = x.w; p[4] = y.x; p[5] = y.y; p[6] = y.z; p[7] = 0.f;
}
template <> __device__ __forceinline__ void load_cell<double>(const StepArgs &a, int64_t c, double p[8])
{
    const double2 *r = reinterpret_cast<const double2 *>(a.params) + 4 * c;
    for (int k = 0; k < 4; ++k) { double2 t = r[k]; p[2 * k] = t.x; p[2 * k + 1] = t.y; }
}

// PRE coupling: site poses, thermal draws, Eq. 7, binning of the sites.
// Arithmetic in the form's precision only (the pose record carries the FP64
// body quantities already reduced to it).
// FP32 site kernels are held to 64 registers (8 CTAs of 128 threads per SM)
// so that they fit beside the solvent pass they overlap with.
template <typename Real> struct SiteMinBlocks { static constexpr int n = sizeof(Real) == 4 ? 8 : 1; };

template <typename Real>
__global__ void __launch_bounds__(SITE_THREADS, SiteMinBlocks<Real>::n) k_sites_pre(StepArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    Real *vt = reinterpret_cast<Real *>(smem_raw);          // [n_sites][3] thermal draws
    __shared__ Real sPose[POSE_W], sVt[3], sWt[3], sred[6];
    __shared__ Real scratch[SITE_WARPS][6];
    __shared__ int sS[3];
    const DevBody &B = a.bodies[blockIdx.x];
    const int shape = B.shape, rep = B.rep;
    const int64_t site_begin = B.site_begin;
    const DevShape sh = a.shapes[shape];
    const DevReplica r = a.reps[rep];
    const int64_t step = *a.d_step + a.step_offset;
    if (threadIdx.x < POSE_W) sPose[threadIdx.x] = pose_ptr(a, blockIdx.x, Real(0))[threadIdx.x];
    if (threadIdx.x == 0) grid_shift(r, step, sS);
    __syncthreads();
    Pose<Real> P;
    for (int k = 0; k < 9; ++k) P.Q[k] = sPose[k];
    for (int k = 0; k < 3; ++k) { P.R[k] = sPose[9 + k]; P.V[k] = sPose[12 + k]; P.W[k] = sPose[15 + k]; }
    const Real kT = (Real)a.kT;
    const int n = sh.n_sites;
    int bad = 0;
    Real acc[6] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t t = sh.site_begin + j, g = site_begin + j;
        Real d[3], x[3];
        site_geom(a, t, P, r, d, x, bad);
        const int c = cell_axis(x[0], sS[0], r.L[0]) +
                      r.L[0] * (cell_axis(x[1], sS[1], r.L[1]) + r.L[1] * cell_axis(x[2], sS[2], r.L[2]));
        a.site_cell[g] = c;
        if (!a.naive) {
            const Real m = site_mass<Real>(a, t);
            Real nn[3];
            normals3(draw(r, step, (uint32_t)(r.site_id_base + (g - r.site_begin)), TAG_SITE, 0u), nn);
            const Real sc = sqrt(kT / m);
            const Real w[3] = {sc * nn[0], sc * nn[1], sc * nn[2]};
            for (int k = 0; k < 3; ++k) vt[3 * j + k] = w[k];
            const Real p[3] = {m * w[0], m * w[1], m * w[2]};
            acc[0] += p[0]; acc[1] += p[1]; acc[2] += p[2];
            acc[3] += d[1] * p[2] - d[2] * p[1];
            acc[4] += d[2] * p[0] - d[0] * p[2];
            acc[5] += d[0] * p[1] - d[1] * p[0];
        }
    }
    block_sum6<Real>(acc, scratch, sred);
    if (threadIdx.x == 0) {
        if (a.naive) {
            for (int k = 0; k < 3; ++k) { sVt[k] = 0; sWt[k] = 0; }
        } else {
            // V~ = sum m v~ / M, omega~ = Q Ihat^-1 Q^T L~
            Real lb[3], wb[3];
            for (int k = 0; k < 3; ++k) sVt[k] = sred[k] / (Real)sh.M;
            for (int k = 0; k < 3; ++k)
                lb[k] = (P.Q[k] * sred[3] + P.Q[3 + k] * sred[4]) + P.Q[6 + k] * sred[5];
            for (int k = 0; k < 3; ++k) wb[k] = sh.Ihat[k] > 0.0 ? lb[k] / (Real)sh.Ihat[k] : Real(0);
            for (int k = 0; k < 3; ++k)
                sWt[k] = (P.Q[3 * k] * wb[0] + P.Q[3 * k + 1] * wb[1]) + P.Q[3 * k + 2] * wb[2];
        }
    }
    __syncthreads();
    const Real dV[3] = {P.V[0] - sVt[0], P.V[1] - sVt[1], P.V[2] - sVt[2]};
    const Real dW[3] = {P.W[0] - sWt[0], P.W[1] - sWt[1], P.W[2] - sWt[2]};
    Real *SV = reinterpret_cast<Real *>(a.site_v);
    const int64_t NS = a.n_sites;
    // uniform trip count: every lane reaches the warp-wide record flush
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool valid = j < n;
        Real v[3] = {0, 0, 0}, xi[3] = {0, 0, 0}, m = Real(0);
        int cell = 0;
        bool own = true;   // a slab bins only the sites in its z range
        if (valid) {
            const int64_t t = sh.site_begin + j, g = site_begin + j;
            Real d[3], x[3];
            site_geom(a, t, P, r, d, x, bad);
            own = site_owned(a, x[2]);
            v[0] = dV[0] + (dW[1] * d[2] - dW[2] * d[1]);
            v[1] = dV[1] + (dW[2] * d[0] - dW[0] * d[2]);
            v[2] = dV[2] + (dW[0] * d[1] - dW[1] * d[0]);
            if (!a.naive)
                for (int k = 0; k < 3; ++k) v[k] += vt[3 * j + k];
            for (int k = 0; k < 3; ++k) SV[k * NS + g] = v[k];
            m = site_mass<Real>(a, t);
            if (a.rule == 1) {
                normals3(draw(r, step, (uint32_t)(r.site_id_base + (g - r.site_begin)), TAG_AT, 0u), xi);
                const Real sc = sqrt(kT / m);
                xi[0] *= sc; xi[1] *= sc; xi[2] *= sc;
            }
            cell = r.cell_base + a.site_cell[g];
        }
        if (valid && own) {
            if constexpr (sizeof(Real) == 4) {
                long long w[MAX_WORDS32];
                unsigned long long *S = reinterpret_cast<unsigned long long *>(a.sums);
                if (a.rule == 0) {
                    record_terms<0>(m, v[0], v[1], v[2], xi, true, w);
                    for (int k = 0; k < Words32<0>::n; ++k)
                        atomicAdd(S + k * a.n_cells + cell, (unsigned long long)w[k]);
                } else {
                    record_terms<1>(m, v[0], v[1], v[2], xi, true, w);
                    for (int k = 0; k < Words32<1>::n; ++k)
                        atomicAdd(S + k * a.n_cells + cell, (unsigned long long)w[k]);
                }
            } else {
                add_sums64(a, cell, m, v, xi);
            }
        }
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// POST coupling: site collision and the per-warp partial sums of the
// momentum dP = sum m (v' - v) and angular momentum dL = sum d x m (v' - v)
// transferred to the body (Eqs. 3-4); k_body_impulse adds them in FP64.
// the collision rule for one site: v -> vn with the parameters p of its cell
template <typename Real>
__device__ __forceinline__ void site_rule(const StepArgs &a, const DevReplica &r, int64_t step, int64_t g,
                                          const Real (&v)[3], const Real (&p)[8], Real m, Real (&vn)[3])
{
    vn[0] = v[0]; vn[1] = v[1]; vn[2] = v[2];
    if (p[3] >= Real(0)) {
        const Real kT = (Real)a.kT, ca = (Real)a.cos_a, sa = (Real)a.sin_a;
        if (a.rule == 0) {
            const Real w[3] = {v[0] - p[0], v[1] - p[1], v[2] - p[2]};
            const Real nd = p[4] * w[0] + p[5] * w[1] + p[6] * w[2];
            const Real cx = p[5] * w[2] - p[6] * w[1], cy = p[6] * w[0] - p[4] * w[2];
            const Real cz = p[4] * w[1] - p[5] * w[0];
            const Real tt = nd * (Real(1) - ca);
            vn[0] = p[0] + p[3] * (w[0] * ca + cx * sa + p[4] * tt);
            vn[1] = p[1] + p[3] * (w[1] * ca + cy * sa + p[5] * tt);
            vn[2] = p[2] + p[3] * (w[2] * ca + cz * sa + p[6] * tt);
        } else {
            Real xi[3];
            normals3(draw(r, step, (uint32_t)(r.site_id_base + (g - r.site_begin)), TAG_AT, 0u), xi);
            const Real sc = sqrt(kT / m);
            for (int k = 0; k < 3; ++k) vn[k] = p[k] + sc * xi[k] - p[4 + k];
        }
    }
}

// lattice offset of a stored site position inside its shifted cell (+a variants)
template <typename Real>
__device__ __forceinline__ void site_lattice_q(const Real (&x)[3], int4 S, int (&Q)[3])
{
    Q[0] = ang_lattice_q(x[0], S.x);
    Q[1] = ang_lattice_q(x[1], S.y);
    Q[2] = ang_lattice_q(x[2], S.z);
}

// POST coupling; ANG: with the +a correction of the site's cell applied to the
// rule's velocity before the momentum change is taken
template <typename Real, bool ANG>
__global__ void __launch_bounds__(SITE_THREADS, SiteMinBlocks<Real>::n) k_sites_post(StepArgs a)
{
    __shared__ Real sPose[POSE_W];
    const DevBody &B = a.bodies[blockIdx.x];
    const int64_t site_begin = B.site_begin;
    const DevShape sh = a.shapes[B.shape];
    const DevReplica r = a.reps[B.rep];
    const int64_t step = *a.d_step;
    if (threadIdx.x < POSE_W) sPose[threadIdx.x] = pose_ptr(a, blockIdx.x, Real(0))[threadIdx.x];
    __syncthreads();
    Pose<Real> P;
    for (int k = 0; k < 9; ++k) P.Q[k] = sPose[k];
    for (int k = 0; k < 3; ++k) { P.R[k] = sPose[9 + k]; P.V[k] = 0; P.W[k] = 0; }
    const Real *SV = reinterpret_cast<const Real *>(a.site_v);
    const int64_t NS = a.n_sites;
    int bad = 0;
    Real acc[6] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < sh.n_sites; j += blockDim.x) {
        const int64_t t = sh.site_begin + j, g = site_begin + j;
        Real d[3], x[3];
        site_geom(a, t, P, r, d, x, bad);
        const Real v[3] = {SV[g], SV[NS + g], SV[2 * NS + g]};
        Real vn[3];
        Real p[8];
        const int64_t cell = (int64_t)r.cell_base + a.site_cell[g];
        load_cell<Real>(a, cell, p);
        const Real m = site_mass<Real>(a, t);
        site_rule<Real>(a, r, step, g, v, p, m, vn);
        if constexpr (ANG) {
            const Real xs[3] = {x[0], x[1], x[2]};
            int Q[3];
            site_lattice_q(xs, a.ang_shift[B.rep], Q);
            ang_correct(reinterpret_cast<const AngParams<Real> *>(a.ang_params)[cell], Q, vn);
        }
        const bool own = site_owned(a, x[2]);   // a slab transfers only its own sites
        const Real dp[3] = {own ? m * (vn[0] - v[0]) : Real(0), own ? m * (vn[1] - v[1]) : Real(0),
                            own ? m * (vn[2] - v[2]) : Real(0)};
        acc[0] += dp[0]; acc[1] += dp[1]; acc[2] += dp[2];
        acc[3] += d[1] * dp[2] - d[2] * dp[1];
        acc[4] += d[2] * dp[0] - d[0] * dp[2];
        acc[5] += d[0] * dp[1] - d[1] * dp[0];
    }
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0) {
        Real *out = reinterpret_cast<Real *>(a.partial) + ((int64_t)blockIdx.x * SITE_WARPS + (threadIdx.x >> 5)) * 6;
        for (int k = 0; k < 6; ++k) out[k] = acc[k];
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

// impulse P += dP, L += dL accumulated in FP64 from the per-warp partials
template <typename Real>
__global__ void k_body_impulse(StepArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const Real *in = reinterpret_cast<const Real *>(a.partial) + (int64_t)i * SITE_WARPS * 6;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < SITE_WARPS; ++w)
        for (int k = 0; k < 6; ++k) s[k] += (double)in[w * 6 + k];
    DevBody *o = a.bodies + i;
    for (int k = 0; k < 3; ++k) {
        o->P[k] += s[k];
        o->Lm[k] += s[3 + k];
    }
}

cudaError_t configure_body_kernels(int max_sites, int precision)
{
    size_t bytes = (size_t)max_sites * 3 * (precision == 1 ? sizeof(float) : sizeof(double));
    if (bytes <= 48 * 1024) return cudaSuccess;
    if (precision == 1)
        return cudaFuncSetAttribute(k_sites_pre<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaFuncSetAttribute(k_sites_pre<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_sites_pre(const StepArgs &a, int max_sites, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    if (a.precision == 1)
        k_sites_pre<float><<<a.n_bodies, SITE_THREADS, (size_t)max_sites * 3 * sizeof(float), s>>>(a);
    else
        k_sites_pre<double><<<a.n_bodies, SITE_THREADS, (size_t)max_sites * 3 * sizeof(double), s>>>(a);
}

void launch_sites_post(const StepArgs &a, int, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    const bool ang = a.ang_params != nullptr;
    if (a.precision == 1) {
        if (ang) k_sites_post<float, true><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
        else k_sites_post<float, false><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
    } else {
        if (ang) k_sites_post<double, true><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
        else k_sites_post<double, false><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
    }
}

// +a variants: the sites' contributions to the angular words of their cells,
// one CTA per body.  PRE: count, sum Q, sum Q_a Q_b, + Q x P, + P from the
// thermalised velocities of Eq. 7; POST: - Q x P*, - P* from the rule's
// velocities (recomputed with the same arithmetic as the POST coupling).
__device__ __forceinline__ long long site_mom_term(float m, float v) { return q20(__fmul_rn(m, v)); }
__device__ __forceinline__ double site_mom_term(double m, double v) { return m * v; }

template <typename Real, bool PRE>
__global__ void __launch_bounds__(SITE_THREADS, SiteMinBlocks<Real>::n) k_ang_sites(StepArgs a)
{
    typedef typename AngWord<Real>::type W;
    __shared__ Real sPose[POSE_W];
    const DevBody &B = a.bodies[blockIdx.x];
    const int64_t site_begin = B.site_begin;
    const DevShape sh = a.shapes[B.shape];
    const DevReplica r = a.reps[B.rep];
    const int64_t step = *a.d_step;
    const int4 S = a.ang_shift[B.rep];
    W *w = reinterpret_cast<W *>(a.ang_words);
    const int64_t C = a.n_cells;
    if (threadIdx.x < POSE_W) sPose[threadIdx.x] = pose_ptr(a, blockIdx.x, Real(0))[threadIdx.x];
    __syncthreads();
    Pose<Real> P;
    for (int k = 0; k < 9; ++k) P.Q[k] = sPose[k];
    for (int k = 0; k < 3; ++k) { P.R[k] = sPose[9 + k]; P.V[k] = 0; P.W[k] = 0; }
    const Real *SV = reinterpret_cast<const Real *>(a.site_v);
    const int64_t NS = a.n_sites;
    int bad = 0;
    for (int j = threadIdx.x; j < sh.n_sites; j += blockDim.x) {
        const int64_t t = sh.site_begin + j, g = site_begin + j;
        Real d[3], x[3];
        site_geom(a, t, P, r, d, x, bad);
        const Real v[3] = {SV[g], SV[NS + g], SV[2 * NS + g]};
        const int64_t cell = (int64_t)r.cell_base + a.site_cell[g];
        const Real m = site_mass<Real>(a, t);
        Real u[3] = {v[0], v[1], v[2]};
        if (!PRE) {
            Real p[8];
            load_cell<Real>(a, cell, p);
            site_rule<Real>(a, r, step, g, v, p, m, u);
        }
        const Real xs[3] = {x[0], x[1], x[2]};
        int Qi[3];
        site_lattice_q(xs, S, Qi);
        const W q[3] = {(W)Qi[0], (W)Qi[1], (W)Qi[2]};
        const W Pm[3] = {(W)site_mom_term(m, u[0]), (W)site_mom_term(m, u[1]), (W)site_mom_term(m, u[2])};
        const W L[3] = {q[1] * Pm[2] - q[2] * Pm[1], q[2] * Pm[0] - q[0] * Pm[2], q[0] * Pm[1] - q[1] * Pm[0]};
        const W sg = PRE ? (W)1 : (W)-1;
        if (PRE) {
            ang_red(w + AW_COUNT * C + cell, (W)4096);
            for (int k = 0; k < 3; ++k) ang_red(w + (AW_SQB + k) * C + cell, q[k]);
            ang_red(w + (AW_QQB + 0) * C + cell, q[0] * q[0]);
            ang_red(w + (AW_QQB + 1) * C + cell, q[1] * q[1]);
            ang_red(w + (AW_QQB + 2) * C + cell, q[2] * q[2]);
            ang_red(w + (AW_QQB + 3) * C + cell, q[0] * q[1]);
            ang_red(w + (AW_QQB + 4) * C + cell, q[0] * q[2]);
            ang_red(w + (AW_QQB + 5) * C + cell, q[1] * q[2]);
        }
        for (int k = 0; k < 3; ++k) {
            ang_red(w + (AW_L + k) * C + cell, sg * L[k]);
            ang_red(w + (AW_P + k) * C + cell, sg * Pm[k]);
        }
    }
    if (bad) atomicOr(a.d_err, ERR_POSITION);
}

void launch_angular_sites(const StepArgs &a, int phase, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    const bool p32 = a.precision == 1;
    if (phase == ANG_PRE) {
        if (p32) k_ang_sites<float, true><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
        else k_ang_sites<double, true><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
    } else if (phase == ANG_POST) {
        if (p32) k_ang_sites<float, false><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
        else k_ang_sites<double, false><<<a.n_bodies, SITE_THREADS, 0, s>>>(a);
    }
}

void launch_body_impulse(const StepArgs &a, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    if (a.precision == 1) k_body_impulse<float><<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a);
    else k_body_impulse<double><<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a);
}

__global__ void k_advance_step(int64_t *step) { *step += 1; }

void launch_advance_step(const StepArgs &a, cudaStream_t s)
{
    k_advance_step<<<1, 1, 0, s>>>(const_cast<int64_t *>(a.d_step));
}

// FP64 body diagnostics: sum P, sum |P|^2/2M, sum L_b.Ihat^-1.L_b/2 (L_b = Q^T L)
__global__ void k_body_diag(StepArgs a, double *acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_bodies) return;
    const DevBody b = a.bodies[i];
    const DevShape sh = a.shapes[b.shape];
    double Lb[3], Q[9];
    rotmat(b.q, Q);
    mtv(Q, b.Lm, Lb);
    double er = 0.0;
    for (int k = 0; k < 3; ++k) er += sh.Ihat[k] > 0.0 ? 0.5 * Lb[k] * Lb[k] / sh.Ihat[k] : 0.0;
    double et = 0.5 * (b.P[0] * b.P[0] + b.P[1] * b.P[1] + b.P[2] * b.P[2]) / sh.M;
    atomicAdd(acc + 4, b.P[0]);
    atomicAdd(acc + 5, b.P[1]);
    atomicAdd(acc + 6, b.P[2]);
    atomicAdd(acc + 7, et);
    atomicAdd(acc + 8, er);
}

void launch_body_diag(const StepArgs &a, double *acc, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    k_body_diag<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a, acc);
}


// ------------------------------------------- velocity autocorrelation
// Sec. III.A: C_T(t) = <V(0).V(t)> and C_R(t) = <omega(0).omega(t)>, every
// sample a time origin.  After every `every`-th completed step each body adds
// V(t).V(t - k) and omega(t).omega(t - k) for the lags k it has samples for;
// the last n_lags samples stay in a per-body ring.  omega is the space-frame
// angular velocity Q Ihat^-1 Q^T L.  FP64, one thread per body.
__global__ void k_vacf_sample(StepArgs a, VacfArgs g)
{
    const int64_t done = *a.d_step + 1 - g.start;   // steps completed since the start
    if (done <= 0 || done % g.every != 0) return;
    const int64_t smp = done / g.every - 1;          // this sample's index
    const int nk = (int)(smp + 1 < g.n_lags ? smp + 1 : g.n_lags);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0)
        for (int k = 0; k < nk; ++k) g.count[k] += 1;
    if (i >= a.n_bodies) return;
    const DevBody b = a.bodies[i];
    const DevShape sh = a.shapes[b.shape];
    double Q[9], Lb[3], wb[3], V[3], W[3];
    rotmat(b.q, Q);
    mtv(Q, b.Lm, Lb);
    for (int k = 0; k < 3; ++k) {
        V[k] = b.P[k] / sh.M;
        wb[k] = sh.Ihat[k] > 0.0 ? Lb[k] / sh.Ihat[k] : 0.0;
    }
    mv(Q, wb, W);
    const int64_t base = (int64_t)i * g.n_lags;
    for (int k = 0; k < nk; ++k) {
        double cv, cw;
        if (k == 0) {
            cv = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
            cw = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
        } else {
            const int64_t r = 3 * (base + (smp - k) % g.n_lags);
            cv = V[0] * g.ring_v[r] + V[1] * g.ring_v[r + 1] + V[2] * g.ring_v[r + 2];
            cw = W[0] * g.ring_w[r] + W[1] * g.ring_w[r + 1] + W[2] * g.ring_w[r + 2];
        }
        g.ct[base + k] += cv;
        g.cr[base + k] += cw;
    }
    const int64_t r = 3 * (base + smp % g.n_lags);
    for (int k = 0; k < 3; ++k) {
        g.ring_v[r + k] = V[k];
        g.ring_w[r + k] = W[k];
    }
}

void launch_vacf_sample(const StepArgs &a, const VacfArgs &g, cudaStream_t s)
{
    if (a.n_bodies == 0) return;
    k_vacf_sample<<<(a.n_bodies + 127) / 128, 128, 0, s>>>(a, g);
}

}  // namespace mpcd
