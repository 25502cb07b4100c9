/*
 * gve_oracle.c -- plain FP64 CPU oracle for fixed-budget Gaussian volume
 * encoding (arxiv 2608.14112).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares
 * no code, header, table or constant generator with the CUDA path; it is
 * written to be read against the paper, not to be fast.
 *
 * What each part follows:
 *   - Primitive parameterisation: Sec. III-C, Eq. 2 (position, log-scales,
 *     normalised quaternion, scalar attribute a, weight w = sigmoid(logit)).
 *   - Field: Sec. III-C, Eq. 3, normalised Gaussian kernel regression with
 *     density floor rho0 and truncation at squared Mahalanobis distance k^2.
 *   - Loss: full-grid mean squared error (Sec. III-E, Eq. 6 value term as a
 *     mean over voxel centres; optional occupancy mask 1[V > thr]).
 *   - PSNR: 10 log10(1/MSE) (Sec. IV-C).
 *   - Gradient: hand-derived chain rule through Eq. 3 and Eq. 2 (the paper's
 *     closed-form-gradient engine, Sec. V-D).
 *   - Adam with bias correction (Sec. III-E, Kingma and Ba).
 *   - Allocation: Sec. III-E (Structure-Aware Fixed-Budget Allocation) and
 *     Table I stages S1a..S1e; Eq. 4 jitter.
 *   - Budget limit: Sec. V-B (seed limit).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Truncation decision.  Whether a (voxel, Gaussian) pair is kept decides
 *     an integer (membership), so it is taken in float32, the paper's
 *     precision: float32 coefficients of -0.5*log2(e)*C are obtained by
 *     rounding an FP64 computation done in a fixed operation order, and the
 *     exponent t is evaluated by a fixed chain of float32 fused multiply-adds;
 *     the pair is kept iff t > T, T = fp32(-0.5*log2(e)*k^2).  The VALUE of
 *     every kept pair is then evaluated in FP64 from the FP64 parameters.
 *   - w = sigmoid(w_logit); the scalar a is a raw parameter.
 *   - Quaternion order (w,x,y,z), normalised in every forward pass.
 *   - Voxel (i,j,k) has its centre at (i,j,k); x is the fastest axis.
 *   - Gradient stencil: central differences, one-sided at the borders.
 *   - Occupancy V > 0.02 decided in float32; detail eligibility adds g > 0.
 *   - Detail/coverage counts Nd = floor(0.55 N + 1/2), Nc = N - Nd.
 *   - Weighted draw without replacement: Efraimidis-Spirakis keys
 *     -ln(u)/g with u from Philox4x32-10 (Salmon et al. 2011); the Nd smallest
 *     keys win, ties broken by voxel index.  The coverage draw keeps the Nc
 *     smallest raw 64-bit Philox words among occupied voxels.
 *   - Jitter u_k = (x_k >> 8) * 2^-24 - 1/2 from Philox (Eq. 4).
 *   - Group spacing: lower median, over an evenly strided subsample of at most
 *     4096 seeds of the group, of the mean distance to the 3 nearest seeds of
 *     the same group; sigma_g = h_g / 2.
 *   - Tangent elongation s_t = sigma_g * clamp(1 + g(c)/gbar, 1, 3), gbar the
 *     lower median of g over occupied voxels; s_perp = sigma_g; all scales
 *     clamped to [0.3, max(nx,ny,nz)/16].
 *   - 7^3 structure-tensor window clipped at the borders; cyclic Jacobi.
 *   - Initial a = trilinear V at mu (edge clamped); w = 0.1.
 *
 * Everything here is FP64 unless a comment says float32.
 */
#include <math.h>
#include <time.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* -0.5 * log2(e): the factor that turns a squared Mahalanobis distance into a
 * base-2 exponent.  Used only for the float32 truncation decision. */
#define OR_NEG_HALF_LOG2E (-0.72134752044448170367996234050095)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.   */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout used by the allocator: (lo32(index), hi32(index), stream,
 * 'GVE1'), key = (lo32(seed), hi32(seed)). */
#define OR_CTR_TAG 0x47564531u
static void or_draw(uint64_t index, uint32_t stream, uint64_t seed, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), stream, OR_CTR_TAG};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Primitive activation, Eq. 2: mu, s = exp(log s), q/|q|, R(q), w, a.       */
/* Record layout: [mux muy muz ls0 ls1 ls2 qw qx qy qz a w_logit].           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double mu[3], s[3], q[4], nq;   /* q normalised, nq = |q_raw| */
    double R[3][3];                 /* rotation of the normalised quaternion */
    double C[3][3];                 /* inverse covariance R diag(s^-2) R^T */
    double w, a;
    int valid;
} act_t;

static void rot_from_quat(double w, double x, double y, double z, double R[3][3])
{
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static int all_finite(const double* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(p[i])) return 0;
    return 1;
}

static void activate(const double* p, act_t* A)
{
    memset(A, 0, sizeof(*A));
    if (!all_finite(p, 12)) return;
    for (int j = 0; j < 3; ++j) { A->mu[j] = p[j]; A->s[j] = exp(p[3 + j]); }
    double qw = p[6], qx = p[7], qy = p[8], qz = p[9];
    double nq = sqrt(((qw * qw + qx * qx) + qy * qy) + qz * qz);
    if (!(nq > 0.0) || !isfinite(nq)) return;
    for (int j = 0; j < 3; ++j)
        if (!(A->s[j] > 0.0) || !isfinite(A->s[j])) return;
    A->nq = nq;
    A->q[0] = qw / nq; A->q[1] = qx / nq; A->q[2] = qy / nq; A->q[3] = qz / nq;
    rot_from_quat(A->q[0], A->q[1], A->q[2], A->q[3], A->R);
    double inv[3];
    for (int j = 0; j < 3; ++j) inv[j] = 1.0 / (A->s[j] * A->s[j]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            A->C[a][b] = ((A->R[a][0] * A->R[b][0]) * inv[0] + (A->R[a][1] * A->R[b][1]) * inv[1])
                       + (A->R[a][2] * A->R[b][2]) * inv[2];
    A->a = p[10];
    A->w = 1.0 / (1.0 + exp(-p[11]));
    A->valid = 1;
}

/* ------------------------------------------------------------------------ */
/* float32 truncation decision: the reading of the squared-Mahalanobis      */
/* cutoff of Sec. III-C taken in float32.                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    float mu[3];
    float qxx, qyy, qzz, qxy2, qxz2, qyz2;
    int valid;
} pred_t;

/* e^x in float32 by a fixed sequence of correctly rounded operations, so
 * that the GPU reproduces it bit for bit: Cody-Waite reduction x = n ln2 + r
 * (ln2 split into a 16-bit head and a tail, |r| <= ln2/2), a degree-7
 * Taylor polynomial of e^r in Horner form with fused multiply-adds, and the
 * exact scaling by 2^n.  Relative error below 2^-22 (pinned against exp). */
static float exp_fixed(float x)
{
    if (x != x) return x;
    if (x > 88.75f) return INFINITY;
    if (x < -103.5f) return 0.0f;
    const float n = rintf(x * 1.44269504f);
    float r = fmaf(-n, 0.693145751953125f, x);
    r = fmaf(-n, 1.42860677e-06f, r);
    float p = 1.98412698e-04f;
    p = fmaf(p, r, 1.38888889e-03f);
    p = fmaf(p, r, 8.33333333e-03f);
    p = fmaf(p, r, 4.16666667e-02f);
    p = fmaf(p, r, 1.66666667e-01f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return ldexpf(p, (int)n);
}

float or_exp_fixed(float x) { return exp_fixed(x); }

/* Coefficients from the float32 parameter record: the activations and
 * -log2(e)/2 Sigma^-1 = -log2(e)/2 R diag(s^-2) R^T in float32, one fixed
 * sequence of correctly rounded operations (the written order, no
 * contraction), the scales by exp_fixed. */
/* The float32 scales s = exp_fixed(log s) and rotation R of the normalised
 * quaternion (Eq. 2), in the written order; 0 for an invalid record
 * (non-finite values, zero quaternion, scales outside float range). */
static int keep_frame(const float* p32, float s[3], float R[3][3])
{
    int ok = 1;
    for (int i = 0; i < 12; ++i) ok = ok && isfinite(p32[i]);
    if (!ok) return 0;
    for (int j = 0; j < 3; ++j) s[j] = exp_fixed(p32[3 + j]);
    const float qw = p32[6], qx = p32[7], qy = p32[8], qz = p32[9];
    const float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    const float nq = sqrtf(n2);
    if (!(nq > 0.0f) || !isfinite(nq)) return 0;
    for (int j = 0; j < 3; ++j)
        if (!(s[j] > 0.0f) || !isfinite(s[j])) return 0;
    const float w = qw / nq, x = qx / nq, y = qy / nq, z = qz / nq;
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
    return 1;
}

static void pred_coeffs(const float* p32, pred_t* P)
{
    for (int j = 0; j < 3; ++j) P->mu[j] = p32[j];
    P->valid = 0;
    float s[3], R[3][3];
    if (!keep_frame(p32, s, R)) return;
    float inv[3];
    for (int j = 0; j < 3; ++j) inv[j] = 1.0f / (s[j] * s[j]);
    const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    float Q[6];
    const float nhl = (float)OR_NEG_HALF_LOG2E;
    for (int q = 0; q < 6; ++q) {
        const int a = ab[q][0], b = ab[q][1];
        const float c = ((R[a][0] * R[b][0]) * inv[0] + (R[a][1] * R[b][1]) * inv[1]) + (R[a][2] * R[b][2]) * inv[2];
        Q[q] = c * nhl;
    }
    P->qxx = Q[0]; P->qyy = Q[1]; P->qzz = Q[2];
    P->qxy2 = 2.0f * Q[3]; P->qxz2 = 2.0f * Q[4]; P->qyz2 = 2.0f * Q[5];
    P->valid = 1;
}

static float pred_threshold(float k)
{
    double k2 = (double)k * (double)k;
    return (float)(k2 * OR_NEG_HALF_LOG2E);
}

/* Exponent t of the kept-pair test, by a fixed float32 chain. */
static float pred_t_of(const pred_t* P, int x, int y, int z)
{
    float dx = (float)x - P->mu[0];
    float dy = (float)y - P->mu[1];
    float dz = (float)z - P->mu[2];
    float e = P->qxz2 * dz;
    float b = fmaf(P->qxy2, dy, e);
    float f = P->qyz2 * dz;
    float g = fmaf(P->qyy, dy, f);
    float hh = P->qzz * dz;
    float dzh = dz * hh;
    float c = fmaf(dy, g, dzh);
    float u = fmaf(P->qxx, dx, b);
    return fmaf(dx, u, c);
}

float or_pred_t(const float* p32, int x, int y, int z)
{
    pred_t P;
    pred_coeffs(p32, &P);
    if (!P.valid) return -INFINITY;
    return pred_t_of(&P, x, y, z);
}

float or_pred_threshold(float k) { return pred_threshold(k); }

/* ------------------------------------------------------------------------ */
/* Enumeration box used by the oracle itself: a generous superset of every   */
/* voxel the float32 decision can keep (k*1.01 + 1/2 standard deviations).    */
/* ------------------------------------------------------------------------ */
static int enum_box(const act_t* A, double k, int truncated, const int dims[3], int lo[3], int hi[3])
{
    if (!A->valid) return 0;
    for (int j = 0; j < 3; ++j) {
        if (!truncated) { lo[j] = 0; hi[j] = dims[j] - 1; continue; }
        double var = 0.0;
        for (int m = 0; m < 3; ++m) var += A->R[j][m] * A->R[j][m] * A->s[m] * A->s[m];
        double r = (k * 1.01) * sqrt(var) + 0.5;
        double l = ceil(A->mu[j] - r), h = floor(A->mu[j] + r);
        if (!(l <= h)) return 0;
        if (l < 0) l = 0;
        if (h > dims[j] - 1) h = dims[j] - 1;
        if (l > h) return 0;
        lo[j] = (int)l; hi[j] = (int)h;
    }
    return 1;
}

static inline int64_t vidx_of(const int dims[3], int x, int y, int z)
{
    return ((int64_t)z * dims[1] + y) * dims[0] + x;
}

/* Mahalanobis distance squared at voxel centre p, FP64. */
static double maha2(const act_t* A, double px, double py, double pz)
{
    double d[3] = {px - A->mu[0], py - A->mu[1], pz - A->mu[2]};
    double m = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m += d[a] * A->C[a][b] * d[b];
    return m;
}

typedef struct {
    act_t A;
    pred_t P;
    int lo[3], hi[3];
    int has_box;
} gctx_t;

static gctx_t* prepare(const double* prm, const double* pred_prm, int64_t n, double k, int truncated,
                       const int dims[3])
{
    gctx_t* G = (gctx_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(gctx_t));
    if (!G) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        activate(prm + 12 * i, &G[i].A);
        const double* pp = pred_prm ? pred_prm + 12 * i : prm + 12 * i;
        float p32[12];
        for (int j = 0; j < 12; ++j) p32[j] = (float)pp[j];
        pred_coeffs(p32, &G[i].P);
        if (pred_prm) {
            /* the box follows the parameters that decide membership */
            act_t Ap;
            activate(pp, &Ap);
            G[i].has_box = G[i].A.valid && enum_box(&Ap, k, truncated, dims, G[i].lo, G[i].hi);
        } else {
            G[i].has_box = enum_box(&G[i].A, k, truncated, dims, G[i].lo, G[i].hi);
        }
        if (!G[i].P.valid) G[i].has_box = 0;
    }
    return G;
}

static int kept(const gctx_t* g, float T, int truncated, int x, int y, int z)
{
    if (!truncated) return 1;
    return pred_t_of(&g->P, x, y, z) > T;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 over a region [r0, r0+rs) of the grid.  num/den/vt have the         */
/* region's size, x fastest.  truncated = 0 evaluates every voxel for every  */
/* Gaussian (the dense sum).  normalized = 0 returns num (plain sum).        */
/* pred_prm (optional) decides membership instead of prm (frozen mask).      */
/* ------------------------------------------------------------------------ */
static int eval_region_prepared(const gctx_t* G, int64_t n, const int r0[3], const int rs[3], float k,
                                double rho0, int normalized, int truncated, double* num, double* den, double* vt)
{
    float T = pred_threshold(k);
    /* Gaussians whose box meets the region, in ascending index order */
    int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nids = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!G[i].has_box) continue;
        int ok = 1;
        for (int j = 0; j < 3; ++j)
            if (G[i].hi[j] < r0[j] || G[i].lo[j] > r0[j] + rs[j] - 1) ok = 0;
        if (ok) ids[nids++] = i;
    }
    int64_t plane = (int64_t)rs[0] * rs[1];
#pragma omp parallel for schedule(dynamic, 1)
    for (int zz = 0; zz < rs[2]; ++zz) {
        int z = r0[2] + zz;
        double* nm = num + plane * zz;
        double* dn = den + plane * zz;
        for (int64_t v = 0; v < plane; ++v) { nm[v] = 0.0; dn[v] = 0.0; }
        for (int64_t t = 0; t < nids; ++t) {
            const gctx_t* g = &G[ids[t]];
            if (z < g->lo[2] || z > g->hi[2]) continue;
            int y0 = g->lo[1] > r0[1] ? g->lo[1] : r0[1];
            int y1 = g->hi[1] < r0[1] + rs[1] - 1 ? g->hi[1] : r0[1] + rs[1] - 1;
            int x0 = g->lo[0] > r0[0] ? g->lo[0] : r0[0];
            int x1 = g->hi[0] < r0[0] + rs[0] - 1 ? g->hi[0] : r0[0] + rs[0] - 1;
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x) {
                    if (!kept(g, T, truncated, x, y, z)) continue;
                    double Gv = exp(-0.5 * maha2(&g->A, x, y, z));
                    int64_t v = (int64_t)(y - r0[1]) * rs[0] + (x - r0[0]);
                    nm[v] += g->A.w * g->A.a * Gv;
                    dn[v] += g->A.w * Gv;
                }
        }
        if (vt) {
            double* o = vt + plane * zz;
            for (int64_t v = 0; v < plane; ++v) {
                if (!normalized) o[v] = nm[v];
                else o[v] = nm[v] / (dn[v] > rho0 ? dn[v] : rho0);
            }
        }
    }
    free(ids);
    return 0;
}

int or_eval_region(const double* prm, const double* pred_prm, int64_t n, const int dims[3],
                   const int r0[3], const int rs[3], float k, double rho0, int normalized,
                   int truncated, double* num, double* den, double* vt)
{
    gctx_t* G = prepare(prm, pred_prm, n, (double)k, truncated, dims);
    if (!G) return 1;
    int rc = eval_region_prepared(G, n, r0, rs, k, rho0, normalized, truncated, num, den, vt);
    free(G);
    return rc;
}

/* Eq. 3 on nblk regions of the same size rs, corners r0s[b][3]: the
 * primitives are activated once for all of them (large models, many small
 * regions).  vt: [nblk][rs[2]][rs[1]][rs[0]]. */
int or_eval_blocks(const double* prm, int64_t n, const int dims[3], int64_t nblk, const int* r0s, const int rs[3],
                   float k, double rho0, int normalized, double* vt)
{
    gctx_t* G = prepare(prm, NULL, n, (double)k, 1, dims);
    if (!G) return 1;
    int64_t R = (int64_t)rs[0] * rs[1] * rs[2];
    double* num = (double*)malloc(sizeof(double) * (size_t)R);
    double* den = (double*)malloc(sizeof(double) * (size_t)R);
    int rc = (num && den) ? 0 : 1;
    for (int64_t b = 0; b < nblk && rc == 0; ++b)
        rc = eval_region_prepared(G, n, r0s + 3 * b, rs, k, rho0, normalized, 1, num, den, vt + R * b);
    free(num); free(den); free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Loss (mean squared error over all M voxel centres, optional occupancy     */
/* mask) and its analytic gradient with respect to the raw 12-float record. */
/* grad may be NULL.  sse_out receives the unmasked sum of squared errors   */
/* (for PSNR = 10 log10(M / sse)).                                          */
/* ------------------------------------------------------------------------ */
static void chain_rule(const act_t* A, const double* raw, double Ag, double Bg, const double S1[3],
                       const double S2[3][3], double* out)
{
    /* dL/da, dL/dw, dL/dw_logit (Eq. 2 sigmoid) */
    double w = A->w, a = A->a;
    out[10] = w * Ag;
    double dw = a * Ag + Bg;
    out[11] = dw * w * (1.0 - w);
    /* dL/dmu = -2 C S1 */
    for (int i = 0; i < 3; ++i) {
        double t = 0.0;
        for (int j = 0; j < 3; ++j) t += A->C[i][j] * S1[j];
        out[i] = -2.0 * t;
    }
    /* C = R D R^T, D = diag(s^-2); dL/dC = S2 (symmetric) */
    double D[3];
    for (int j = 0; j < 3; ++j) D[j] = 1.0 / (A->s[j] * A->s[j]);
    /* dL/dD_jj = (R^T S2 R)_jj ; dD_jj/dlog s_j = -2 D_jj */
    for (int j = 0; j < 3; ++j) {
        double t = 0.0;
        for (int a2 = 0; a2 < 3; ++a2)
            for (int b = 0; b < 3; ++b) t += A->R[a2][j] * S2[a2][b] * A->R[b][j];
        out[3 + j] = -2.0 * D[j] * t;
    }
    /* dL/dR = 2 S2 R D */
    double gR[3][3];
    for (int a2 = 0; a2 < 3; ++a2)
        for (int j = 0; j < 3; ++j) {
            double t = 0.0;
            for (int b = 0; b < 3; ++b) t += S2[a2][b] * A->R[b][j];
            gR[a2][j] = 2.0 * t * D[j];
        }
    /* dR/dq_hat for R(q) written out entry by entry */
    double qw = A->q[0], qx = A->q[1], qy = A->q[2], qz = A->q[3];
    double gw = 0, gx = 0, gy = 0, gz = 0;
    /* R00 = 1-2y^2-2z^2 */
    gy += gR[0][0] * (-4.0 * qy); gz += gR[0][0] * (-4.0 * qz);
    /* R01 = 2xy - 2wz */
    gw += gR[0][1] * (-2.0 * qz); gx += gR[0][1] * (2.0 * qy); gy += gR[0][1] * (2.0 * qx); gz += gR[0][1] * (-2.0 * qw);
    /* R02 = 2xz + 2wy */
    gw += gR[0][2] * (2.0 * qy); gx += gR[0][2] * (2.0 * qz); gy += gR[0][2] * (2.0 * qw); gz += gR[0][2] * (2.0 * qx);
    /* R10 = 2xy + 2wz */
    gw += gR[1][0] * (2.0 * qz); gx += gR[1][0] * (2.0 * qy); gy += gR[1][0] * (2.0 * qx); gz += gR[1][0] * (2.0 * qw);
    /* R11 = 1-2x^2-2z^2 */
    gx += gR[1][1] * (-4.0 * qx); gz += gR[1][1] * (-4.0 * qz);
    /* R12 = 2yz - 2wx */
    gw += gR[1][2] * (-2.0 * qx); gx += gR[1][2] * (-2.0 * qw); gy += gR[1][2] * (2.0 * qz); gz += gR[1][2] * (2.0 * qy);
    /* R20 = 2xz - 2wy */
    gw += gR[2][0] * (-2.0 * qy); gx += gR[2][0] * (2.0 * qz); gy += gR[2][0] * (-2.0 * qw); gz += gR[2][0] * (2.0 * qx);
    /* R21 = 2yz + 2wx */
    gw += gR[2][1] * (2.0 * qx); gx += gR[2][1] * (2.0 * qw); gy += gR[2][1] * (2.0 * qz); gz += gR[2][1] * (2.0 * qy);
    /* R22 = 1-2x^2-2y^2 */
    gx += gR[2][2] * (-4.0 * qx); gy += gR[2][2] * (-4.0 * qy);
    /* through q_hat = q / |q| */
    double dot = gw * qw + gx * qx + gy * qy + gz * qz;
    out[6] = (gw - qw * dot) / A->nq;
    out[7] = (gx - qx * dot) / A->nq;
    out[8] = (gy - qy * dot) / A->nq;
    out[9] = (gz - qz * dot) / A->nq;
    (void)raw;
}

/* Per-Gaussian sums over its kept voxels given dL/dnum (gn) and dL/dden (gd)
 * per voxel, then the chain rule to the raw record. */
static void accumulate_grads(const double* prm, const double* pred_prm, int64_t n, const int dims[3], float k,
                             int truncated, const double* gn, const double* gd, double* grad)
{
    gctx_t* G = prepare(prm, pred_prm, n, (double)k, truncated, dims);
    float T = pred_threshold(k);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double* out = grad + 12 * i;
        for (int j = 0; j < 12; ++j) out[j] = 0.0;
        const gctx_t* g = &G[i];
        if (!g->has_box || !g->A.valid) continue;
        double Ag = 0, Bg = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0}};
        for (int z = g->lo[2]; z <= g->hi[2]; ++z)
            for (int y = g->lo[1]; y <= g->hi[1]; ++y)
                for (int x = g->lo[0]; x <= g->hi[0]; ++x) {
                    if (!kept(g, T, truncated, x, y, z)) continue;
                    int64_t v = ((int64_t)z * dims[1] + y) * dims[0] + x;
                    double d[3] = {x - g->A.mu[0], y - g->A.mu[1], z - g->A.mu[2]};
                    double Gv = exp(-0.5 * maha2(&g->A, x, y, z));
                    Ag += Gv * gn[v];
                    Bg += Gv * gd[v];
                    double c = g->A.w * (g->A.a * gn[v] + gd[v]);   /* dL/dG */
                    double h = -0.5 * c * Gv;                        /* dL/dm */
                    for (int a2 = 0; a2 < 3; ++a2) {
                        S1[a2] += h * d[a2];
                        for (int b = 0; b < 3; ++b) S2[a2][b] += h * d[a2] * d[b];
                    }
                }
        chain_rule(&g->A, prm + 12 * i, Ag, Bg, S1, S2, out);
    }
    free(G);
}

double or_loss_grad(const double* prm, const double* pred_prm, int64_t n, const float* field,
                    const int dims[3], float k, double rho0, int normalized, int truncated,
                    double mask_thresh, double* grad, double* sse_out)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2];
    int r0[3] = {0, 0, 0};
    double* num = (double*)malloc(sizeof(double) * (size_t)M);
    double* den = (double*)malloc(sizeof(double) * (size_t)M);
    double* vt = (double*)malloc(sizeof(double) * (size_t)M);
    double* gn = grad ? (double*)malloc(sizeof(double) * (size_t)M) : NULL;
    double* gd = grad ? (double*)malloc(sizeof(double) * (size_t)M) : NULL;
    if (!num || !den || !vt || (grad && (!gn || !gd))) return NAN;
    or_eval_region(prm, pred_prm, n, dims, r0, dims, k, rho0, normalized, truncated, num, den, vt);
    double loss = 0.0, sse = 0.0;
    float mthr = (float)mask_thresh;
    for (int64_t v = 0; v < M; ++v) {
        double r = vt[v] - (double)field[v];
        sse += r * r;
        int in = mask_thresh < 0.0 || field[v] > mthr;
        double rl = in ? r : 0.0;
        loss += rl * rl;
        if (grad) {
            double up = 2.0 * rl / (double)M;           /* dL/dVtilde */
            if (!normalized) { gn[v] = up; gd[v] = 0.0; }
            else if (den[v] >= rho0) { gn[v] = up / den[v]; gd[v] = -vt[v] * gn[v]; }
            else { gn[v] = up / rho0; gd[v] = 0.0; }
        }
    }
    loss /= (double)M;
    if (sse_out) *sse_out = sse;
    if (grad) accumulate_grads(prm, pred_prm, n, dims, k, truncated, gn, gd, grad);
    free(num); free(den); free(vt); free(gn); free(gd);
    return loss;
}

/* Gradient for an arbitrary upstream dL/dVtilde per voxel (the backward of
 * the field evaluation alone). */
int or_backward(const double* prm, int64_t n, const double* upstream, const int dims[3], float k, double rho0,
                int normalized, double* grad)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2];
    int r0[3] = {0, 0, 0};
    double* num = (double*)malloc(sizeof(double) * (size_t)M);
    double* den = (double*)malloc(sizeof(double) * (size_t)M);
    double* vt = (double*)malloc(sizeof(double) * (size_t)M);
    double* gn = (double*)malloc(sizeof(double) * (size_t)M);
    double* gd = (double*)malloc(sizeof(double) * (size_t)M);
    if (!num || !den || !vt || !gn || !gd) return 1;
    or_eval_region(prm, NULL, n, dims, r0, dims, k, rho0, normalized, 1, num, den, vt);
    for (int64_t v = 0; v < M; ++v) {
        double up = upstream[v];
        if (!normalized) { gn[v] = up; gd[v] = 0.0; }
        else if (den[v] >= rho0) { gn[v] = up / den[v]; gd[v] = -vt[v] * gn[v]; }
        else { gn[v] = up / rho0; gd[v] = 0.0; }
    }
    accumulate_grads(prm, NULL, n, dims, k, 1, gn, gd, grad);
    free(num); free(den); free(vt); free(gn); free(gd);
    return 0;
}

/* Number of kept (voxel, Gaussian) pairs: the algorithmic work of one
 * truncated evaluation. */
int64_t or_count_kept(const float* p32, int64_t n, const int dims[3], float k)
{
    float T = pred_threshold(k);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        double p[12];
        for (int j = 0; j < 12; ++j) p[j] = (double)p32[12 * i + j];
        gctx_t g;
        activate(p, &g.A);
        pred_coeffs(p32 + 12 * i, &g.P);
        if (!g.A.valid || !g.P.valid || !enum_box(&g.A, k, 1, dims, g.lo, g.hi)) continue;
        for (int z = g.lo[2]; z <= g.hi[2]; ++z)
            for (int y = g.lo[1]; y <= g.hi[1]; ++y)
                for (int x = g.lo[0]; x <= g.hi[0]; ++x) total += pred_t_of(&g.P, x, y, z) > T;
    }
    return total;
}

/* The kept (voxel, Gaussian) pairs themselves, Gaussian-major, voxels
 * ascending within a Gaussian: out[j] = (voxel index << 24) | Gaussian index
 * for j < min(total, cap).  Returns the total. */
int64_t or_list_kept(const float* p32, int64_t n, const int dims[3], float k, uint64_t* out, int64_t cap)
{
    float T = pred_threshold(k);
    int64_t* cnt = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cnt) return -1;
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double p[12];
            for (int j = 0; j < 12; ++j) p[j] = (double)p32[12 * i + j];
            gctx_t g;
            activate(p, &g.A);
            pred_coeffs(p32 + 12 * i, &g.P);
            if (!g.A.valid || !g.P.valid || !enum_box(&g.A, k, 1, dims, g.lo, g.hi)) continue;
            int64_t m = pass == 0 ? 0 : cnt[i];
            for (int z = g.lo[2]; z <= g.hi[2]; ++z)
                for (int y = g.lo[1]; y <= g.hi[1]; ++y)
                    for (int x = g.lo[0]; x <= g.hi[0]; ++x) {
                        if (!(pred_t_of(&g.P, x, y, z) > T)) continue;
                        if (pass == 1 && m < cap) out[m] = ((uint64_t)vidx_of(dims, x, y, z) << 24) | (uint64_t)i;
                        ++m;
                    }
            if (pass == 0) cnt[i] = m;
        }
        if (pass == 0) {  /* exclusive scan of the per-Gaussian counts */
            int64_t run = 0;
            for (int64_t i = 0; i < n; ++i) { int64_t c = cnt[i]; cnt[i] = run; run += c; }
            cnt[n] = run;
        }
    }
    int64_t total = cnt[n];
    free(cnt);
    return total;
}

/* Gradient for a subset of Gaussians only; the field values it needs are
 * computed on each Gaussian's own box from all Gaussians.  M is the full grid
 * size used as the loss normaliser. */
int or_grad_subset(const double* prm, int64_t n, const float* field, const int dims[3], float k,
                   double rho0, int normalized, double mask_thresh, const int64_t* ids,
                   int64_t nids, double* grad)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2];
    float T = pred_threshold(k);
    float mthr = (float)mask_thresh;
    gctx_t* GA = prepare(prm, NULL, n, (double)k, 1, dims);
    if (!GA) return 1;
    for (int64_t t = 0; t < nids; ++t) {
        int64_t i = ids[t];
        double* out = grad + 12 * t;
        for (int j = 0; j < 12; ++j) out[j] = 0.0;
        gctx_t g;
        activate(prm + 12 * i, &g.A);
        float p32[12];
        for (int j = 0; j < 12; ++j) p32[j] = (float)prm[12 * i + j];
        pred_coeffs(p32, &g.P);
        if (!g.A.valid || !g.P.valid || !enum_box(&g.A, k, 1, dims, g.lo, g.hi)) continue;
        int rs[3] = {g.hi[0] - g.lo[0] + 1, g.hi[1] - g.lo[1] + 1, g.hi[2] - g.lo[2] + 1};
        int64_t R = (int64_t)rs[0] * rs[1] * rs[2];
        double* num = (double*)malloc(sizeof(double) * (size_t)R);
        double* den = (double*)malloc(sizeof(double) * (size_t)R);
        double* vt = (double*)malloc(sizeof(double) * (size_t)R);
        eval_region_prepared(GA, n, g.lo, rs, k, rho0, normalized, 1, num, den, vt);
        double Ag = 0, Bg = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0}};
        for (int z = g.lo[2]; z <= g.hi[2]; ++z)
            for (int y = g.lo[1]; y <= g.hi[1]; ++y)
                for (int x = g.lo[0]; x <= g.hi[0]; ++x) {
                    if (!(pred_t_of(&g.P, x, y, z) > T)) continue;
                    int64_t rv = ((int64_t)(z - g.lo[2]) * rs[1] + (y - g.lo[1])) * rs[0] + (x - g.lo[0]);
                    int64_t v = ((int64_t)z * dims[1] + y) * dims[0] + x;
                    double r = vt[rv] - (double)field[v];
                    if (!(mask_thresh < 0.0 || field[v] > mthr)) r = 0.0;
                    double up = 2.0 * r / (double)M, gnv, gdv;
                    if (!normalized) { gnv = up; gdv = 0.0; }
                    else if (den[rv] >= rho0) { gnv = up / den[rv]; gdv = -vt[rv] * gnv; }
                    else { gnv = up / rho0; gdv = 0.0; }
                    double d[3] = {x - g.A.mu[0], y - g.A.mu[1], z - g.A.mu[2]};
                    double Gv = exp(-0.5 * maha2(&g.A, x, y, z));
                    Ag += Gv * gnv;
                    Bg += Gv * gdv;
                    double c = g.A.w * (g.A.a * gnv + gdv);
                    double h = -0.5 * c * Gv;
                    for (int a2 = 0; a2 < 3; ++a2) {
                        S1[a2] += h * d[a2];
                        for (int b = 0; b < 3; ++b) S2[a2][b] += h * d[a2] * d[b];
                    }
                }
        chain_rule(&g.A, prm + 12 * i, Ag, Bg, S1, S2, out);
        free(num); free(den); free(vt);
    }
    free(GA);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma and Ba 2015) with bias correction; t is 1-based.             */
/* ------------------------------------------------------------------------ */
void or_adam(double* p, double* m, double* v, const double* g, int64_t cnt, int t, double lr,
             double b1, double b2, double eps)
{
    double bc1 = 1.0 - pow(b1, (double)t);
    double bc2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < cnt; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Fixed-budget refinement (Sec. III-E): iters steps of loss -> gradient ->
 * Adam; losses[t] is the loss at the parameters before step t+1; the
 * returned value is the unmasked SSE of one extra evaluation after the last
 * step.  prm is updated in place; m and v (12n each) start at zero. */
double or_refine(double* prm, int64_t n, const float* field, const int dims[3], float k, double rho0,
                 int normalized, double mask_thresh, int iters, double lr, double b1, double b2,
                 double eps, double* losses)
{
    double* g = (double*)malloc(sizeof(double) * 12 * (size_t)(n > 0 ? n : 1));
    double* m = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    double* v = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    for (int t = 0; t < iters; ++t) {
        double sse;
        double L = or_loss_grad(prm, NULL, n, field, dims, k, rho0, normalized, 1, mask_thresh, g, &sse);
        if (losses) losses[t] = L;
        or_adam(prm, m, v, g, 12 * n, t + 1, lr, b1, b2, eps);
    }
    double sse = 0.0;
    or_loss_grad(prm, NULL, n, field, dims, k, rho0, normalized, 1, mask_thresh, NULL, &sse);
    free(g); free(m); free(v);
    return sse;
}

/* ------------------------------------------------------------------------ */
/* Brick binning: which bricks of B^3 voxels may hold a kept pair of         */
/* Gaussian i.  A conservative rule, decided bit-identically on both sides,  */
/* in float32 from the keep test's own scales and rotation (keep_frame):     */
/* a box of Mahalanobis radius kb = k (1.0001 + 1e-5 cond) plus 0.01 voxel,  */
/* then a whitened-distance lower bound per brick.  The relative margins    */
/* (1e-4 + 1e-5 cond) exceed the float32 rounding of the box, of the        */
/* rotation's departure from orthonormality and of the keep chain (a few    */
/* ulps times cond); the 0.01 voxel exceeds the rounding of mu -/+ r and of */
/* brick-centre offsets below 2^14.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int blo[3], bhi[3];
    float L[3][3];
    float e[3];
    float K2;
    int nonempty;
} binspec_t;

static void bin_spec(const float* p32, const int dims[3], float k, int B, binspec_t* S)
{
    memset(S, 0, sizeof(*S));
    float s[3], R[3][3];
    if (!keep_frame(p32, s, R)) return;
    float smin = s[0], smax = s[0];
    for (int j = 1; j < 3; ++j) { if (s[j] < smin) smin = s[j]; if (s[j] > smax) smax = s[j]; }
    float ratio = smax / smin;
    float cond = ratio * ratio;
    float kb = k * (1.0001f + 1e-5f * cond);
    if (!isfinite(kb)) return;
    for (int j = 0; j < 3; ++j) {
        float var = ((R[j][0] * R[j][0]) * (s[0] * s[0]) + (R[j][1] * R[j][1]) * (s[1] * s[1]))
                  + (R[j][2] * R[j][2]) * (s[2] * s[2]);
        float r = kb * sqrtf(var) + 0.01f;
        float l = ceilf(p32[j] - r), h = floorf(p32[j] + r);
        if (!(l <= h) || !isfinite(l) || !isfinite(h)) return;
        if (l < 0.0f) l = 0.0f;
        if (h > (float)(dims[j] - 1)) h = (float)(dims[j] - 1);
        if (l > h) return;
        S->blo[j] = (int)l / B;
        S->bhi[j] = (int)h / B;
    }
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) S->L[j][i] = R[i][j] / s[j];
    float hB = (float)(0.5 * (double)(B - 1)) + 0.01f;
    for (int j = 0; j < 3; ++j) {
        float sabs = (fabsf(S->L[j][0]) + fabsf(S->L[j][1])) + fabsf(S->L[j][2]);
        S->e[j] = hB * sabs;
    }
    S->K2 = (kb * kb) * 1.0001f + 1e-4f;
    S->nonempty = 1;
}

static int bin_test(const binspec_t* S, const float mu[3], int B, int bx, int by, int bz)
{
    float half = (float)(0.5 * (double)(B - 1));
    float cx = (float)(bx * B) + half;
    float cy = (float)(by * B) + half;
    float cz = (float)(bz * B) + half;
    float dcx = cx - mu[0], dcy = cy - mu[1], dcz = cz - mu[2];
    float acc[3];
    for (int j = 0; j < 3; ++j) {
        float t0 = S->L[j][0] * dcx;
        float y = fmaf(S->L[j][2], dcz, fmaf(S->L[j][1], dcy, t0));
        float a = fabsf(y) - S->e[j];
        acc[j] = a > 0.0f ? a : 0.0f;
    }
    float a22 = acc[2] * acc[2];
    float s = fmaf(acc[0], acc[0], fmaf(acc[1], acc[1], a22));
    return s <= S->K2;
}

/* counts[i] = number of bricks listed for Gaussian i; returns the total. */
int64_t or_bin_count(const float* p32, int64_t n, const int dims[3], float k, int B, uint32_t* counts)
{
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        binspec_t S;
        bin_spec(p32 + 12 * i, dims, k, B, &S);
        uint32_t c = 0;
        if (S.nonempty)
            for (int bz = S.blo[2]; bz <= S.bhi[2]; ++bz)
                for (int by = S.blo[1]; by <= S.bhi[1]; ++by)
                    for (int bx = S.blo[0]; bx <= S.bhi[0]; ++bx)
                        c += (uint32_t)bin_test(&S, p32 + 12 * i, B, bx, by, bz);
        counts[i] = c;
        total += c;
    }
    return total;
}

/* (brick key, gid) pairs in Gaussian-major order, bricks z-major within a
 * Gaussian; key = (bz * nby + by) * nbx + bx. */
int64_t or_bin_emit(const float* p32, int64_t n, const int dims[3], float k, int B, uint32_t* keys,
                    uint32_t* gids)
{
    int nbx = (dims[0] + B - 1) / B, nby = (dims[1] + B - 1) / B;
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        binspec_t S;
        bin_spec(p32 + 12 * i, dims, k, B, &S);
        if (!S.nonempty) continue;
        for (int bz = S.blo[2]; bz <= S.bhi[2]; ++bz)
            for (int by = S.blo[1]; by <= S.bhi[1]; ++by)
                for (int bx = S.blo[0]; bx <= S.bhi[0]; ++bx)
                    if (bin_test(&S, p32 + 12 * i, B, bx, by, bz)) {
                        keys[o] = (uint32_t)(((int64_t)bz * nby + by) * nbx + bx);
                        gids[o] = (uint32_t)i;
                        ++o;
                    }
    }
    return o;
}

/* Sub-bricks of listed bricks that hold kept pairs: for pair i (Gaussian
 * gids[i], brick keys[i] of edge B), bit s = (y half) + 2 (z quarter) of
 * masks[i] is set when a voxel centre of the B x B/2 x B/4 sub-brick s,
 * inside the grid and the Gaussian's enumeration box, passes the float32
 * keep test.  The evaluator's sub-brick masks must contain these bits. */
void or_kept_submasks(const float* p32, const int dims[3], float k, int B, int64_t npairs, const uint32_t* keys,
                      const uint32_t* gids, uint8_t* masks)
{
    const float T = pred_threshold(k);
    const int nbx = (dims[0] + B - 1) / B, nby = (dims[1] + B - 1) / B;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < npairs; ++i) {
        const float* r = p32 + 12 * (int64_t)gids[i];
        double p[12];
        for (int j = 0; j < 12; ++j) p[j] = (double)r[j];
        gctx_t g;
        activate(p, &g.A);
        pred_coeffs(r, &g.P);
        uint8_t m = 0;
        if (g.A.valid && g.P.valid && enum_box(&g.A, k, 1, dims, g.lo, g.hi)) {
            const int64_t key = keys[i];
            const int bx = (int)(key % nbx), by = (int)((key / nbx) % nby), bz = (int)(key / ((int64_t)nbx * nby));
            for (int zz = 0; zz < B; ++zz)
                for (int yy = 0; yy < B; ++yy)
                    for (int xx = 0; xx < B; ++xx) {
                        const int x = bx * B + xx, y = by * B + yy, z = bz * B + zz;
                        if (x < g.lo[0] || x > g.hi[0] || y < g.lo[1] || y > g.hi[1] || z < g.lo[2] || z > g.hi[2])
                            continue;
                        if (pred_t_of(&g.P, x, y, z) > T) m |= (uint8_t)(1u << ((yy / (B / 2)) + 2 * (zz / (B / 4))));
                    }
        }
        masks[i] = m;
    }
}

/* ------------------------------------------------------------------------ */
/* Stage P (Sec. III-B): the field rescaled to [0, 1] by its own minimum and */
/* maximum, in float32: out = (V - min) / (max - min), each operation        */
/* correctly rounded (a constant field maps to 0).  minmax (optional)        */
/* receives the two float32 extremes.  Returns 1 (nothing written) when a   */
/* value is not finite, else 0.  out may equal V.                           */
/* ------------------------------------------------------------------------ */
int or_normalize(const float* V, int64_t M, float* out, float* minmax)
{
    if (M <= 0) return 0;
    float mn = V[0], mx = V[0];
    for (int64_t i = 0; i < M; ++i) {
        if (!isfinite(V[i])) return 1;
        if (V[i] < mn) mn = V[i];
        if (V[i] > mx) mx = V[i];
    }
    float range = mx - mn;
    for (int64_t i = 0; i < M; ++i) {
        float d = V[i] - mn;
        out[i] = range > 0.0f ? d / range : 0.0f;
    }
    if (minmax) { minmax[0] = mn; minmax[1] = mx; }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Allocation (Sec. III-E, Table I S1a..S1e).                                */
/* ------------------------------------------------------------------------ */
static inline int64_t vidx(const int dims[3], int x, int y, int z)
{
    return ((int64_t)z * dims[1] + y) * dims[0] + x;
}

/* S1a: float32 gradient magnitude (central differences, one-sided at the
 * borders), in a fixed operation order: the value that decides eligibility
 * and weights the detail draw. */
static float dcomp32(const float* V, const int dims[3], int x, int y, int z, int axis)
{
    int c[3] = {x, y, z};
    int n = dims[axis];
    if (n < 2) return 0.0f;
    int lo = c[axis] - 1, hi = c[axis] + 1;
    float scale = 0.5f;
    if (lo < 0) { lo = c[axis]; scale = 1.0f; }
    if (hi > n - 1) { hi = c[axis]; scale = 1.0f; }
    int a[3] = {x, y, z}, b[3] = {x, y, z};
    a[axis] = hi; b[axis] = lo;
    float diff = V[vidx(dims, a[0], a[1], a[2])] - V[vidx(dims, b[0], b[1], b[2])];
    return scale * diff;
}

static float gmag32_at(const float* V, const int dims[3], int x, int y, int z)
{
    float gx = dcomp32(V, dims, x, y, z, 0);
    float gy = dcomp32(V, dims, x, y, z, 1);
    float gz = dcomp32(V, dims, x, y, z, 2);
    float sx = gx * gx, sy = gy * gy, sz = gz * gz;
    float s = sx + sy;
    s = s + sz;
    return sqrtf(s);
}

void or_grad_mag32(const float* V, const int dims[3], float* g)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < dims[2]; ++z)
        for (int y = 0; y < dims[1]; ++y)
            for (int x = 0; x < dims[0]; ++x) g[vidx(dims, x, y, z)] = gmag32_at(V, dims, x, y, z);
}

/* The same float32 |grad V| at n listed voxel indices. */
void or_grad_mag32_at(const float* V, const int dims[3], const int64_t* vox, int64_t n, float* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = vox[i];
        int x = (int)(v % dims[0]), y = (int)((v / dims[0]) % dims[1]), z = (int)(v / ((int64_t)dims[0] * dims[1]));
        out[i] = gmag32_at(V, dims, x, y, z);
    }
}

/* FP64 gradient vector for the structure tensor. */
static void grad64(const float* V, const int dims[3], int x, int y, int z, double gv[3])
{
    int c[3] = {x, y, z};
    for (int axis = 0; axis < 3; ++axis) {
        int n = dims[axis];
        if (n < 2) { gv[axis] = 0.0; continue; }
        int lo = c[axis] - 1, hi = c[axis] + 1;
        double scale = 0.5;
        if (lo < 0) { lo = c[axis]; scale = 1.0; }
        if (hi > n - 1) { hi = c[axis]; scale = 1.0; }
        int a[3] = {x, y, z}, b[3] = {x, y, z};
        a[axis] = hi; b[axis] = lo;
        gv[axis] = scale * ((double)V[vidx(dims, a[0], a[1], a[2])] - (double)V[vidx(dims, b[0], b[1], b[2])]);
    }
}

/* S1d: 7^3 structure tensor J = sum grad grad^T, window clipped at borders.
 * J6 = [Jxx Jyy Jzz Jxy Jxz Jyz]. */
void or_struct_tensor(const float* V, const int dims[3], int cx, int cy, int cz, double* J6)
{
    double J[6] = {0, 0, 0, 0, 0, 0};
    for (int z = cz - 3; z <= cz + 3; ++z) {
        if (z < 0 || z >= dims[2]) continue;
        for (int y = cy - 3; y <= cy + 3; ++y) {
            if (y < 0 || y >= dims[1]) continue;
            for (int x = cx - 3; x <= cx + 3; ++x) {
                if (x < 0 || x >= dims[0]) continue;
                double g[3];
                grad64(V, dims, x, y, z, g);
                J[0] += g[0] * g[0]; J[1] += g[1] * g[1]; J[2] += g[2] * g[2];
                J[3] += g[0] * g[1]; J[4] += g[0] * g[2]; J[5] += g[1] * g[2];
            }
        }
    }
    memcpy(J6, J, sizeof(J));
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix.  On return
 * evals ascending, evecs columns (evecs[r][c] = component r of vector c). */
void or_jacobi3(const double* J6, double* evals, double* evecs9)
{
    double a[3][3] = {{J6[0], J6[3], J6[4]}, {J6[3], J6[1], J6[5]}, {J6[4], J6[5], J6[2]}};
    double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double fro = off * 2 + a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-30 * fro || off == 0.0) break;
        static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int r = 0; r < 3; ++r) {
            int p = PQ[r][0], q = PQ[r][1];
            if (a[p][q] == 0.0) continue;
            /* rotation that zeroes a[p][q]: tan of the angle solves
             * t^2 + 2 theta t - 1 = 0, smaller root */
            double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            for (int k = 0; k < 3; ++k) {  /* A <- A G (columns p,q) */
                double akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - s * akq;
                a[k][q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {  /* A <- G^T A (rows p,q) */
                double apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - s * aqk;
                a[q][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    /* sort ascending (stable on index for equal eigenvalues) */
    int idx[3] = {0, 1, 2};
    double lam[3] = {a[0][0], a[1][1], a[2][2]};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[idx[j]] < lam[idx[i]] || (lam[idx[j]] == lam[idx[i]] && idx[j] < idx[i])) {
                int t = idx[i]; idx[i] = idx[j]; idx[j] = t;
            }
    for (int c = 0; c < 3; ++c) {
        evals[c] = lam[idx[c]];
        for (int r = 0; r < 3; ++r) evecs9[r * 3 + c] = v[r][idx[c]];
    }
}

/* Quaternion (w,x,y,z), w >= 0, of a proper rotation matrix (Shepperd 1978). */
void or_quat_from_R(const double* R9, double* q)
{
    double R[3][3];
    for (int i = 0; i < 9; ++i) R[i / 3][i % 3] = R9[i];
    double tr = R[0][0] + R[1][1] + R[2][2];
    double w, x, y, z;
    if (tr > 0.0) {
        double S = sqrt(tr + 1.0) * 2.0;
        w = 0.25 * S; x = (R[2][1] - R[1][2]) / S; y = (R[0][2] - R[2][0]) / S; z = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double S = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2.0;
        w = (R[2][1] - R[1][2]) / S; x = 0.25 * S; y = (R[0][1] + R[1][0]) / S; z = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        double S = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2.0;
        w = (R[0][2] - R[2][0]) / S; x = (R[0][1] + R[1][0]) / S; y = 0.25 * S; z = (R[1][2] + R[2][1]) / S;
    } else {
        double S = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2.0;
        w = (R[1][0] - R[0][1]) / S; x = (R[0][2] + R[2][0]) / S; y = (R[1][2] + R[2][1]) / S; z = 0.25 * S;
    }
    if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
    q[0] = w; q[1] = x; q[2] = y; q[3] = z;
}

/* Canonical frame from ascending eigenvectors: e1 (tangent), e2 with their
 * largest-magnitude component made positive, e3 = e1 x e2. R9 columns. */
static void canonical_frame(const double* ev9, double* R9)
{
    double e[2][3];
    for (int c = 0; c < 2; ++c) {
        int best = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(ev9[r * 3 + c]) > fabs(ev9[best * 3 + c])) best = r;
        double sgn = ev9[best * 3 + c] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) e[c][r] = sgn * ev9[r * 3 + c];
    }
    double e3[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                    e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    for (int r = 0; r < 3; ++r) { R9[r * 3 + 0] = e[0][r]; R9[r * 3 + 1] = e[1][r]; R9[r * 3 + 2] = e3[r]; }
}

void or_canonical_frame(const double* ev9, double* R9) { canonical_frame(ev9, R9); }

/* Trilinear interpolation of V at a continuous voxel-index position,
 * coordinates clamped to the grid. */
double or_trilinear(const float* V, const int dims[3], double px, double py, double pz)
{
    double p[3] = {px, py, pz};
    int i0[3], i1[3];
    double f[3];
    for (int j = 0; j < 3; ++j) {
        double c = p[j];
        if (c < 0.0) c = 0.0;
        if (c > dims[j] - 1) c = dims[j] - 1;
        double fl = floor(c);
        i0[j] = (int)fl;
        i1[j] = i0[j] + 1 < dims[j] ? i0[j] + 1 : i0[j];
        f[j] = c - fl;
    }
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double wgt = (cx ? f[0] : 1 - f[0]) * (cy ? f[1] : 1 - f[1]) * (cz ? f[2] : 1 - f[2]);
                acc += wgt * (double)V[vidx(dims, cx ? i1[0] : i0[0], cy ? i1[1] : i0[1], cz ? i1[2] : i0[2])];
            }
    return acc;
}

/* Largest budget N' <= N whose detail and coverage draws both fit
 * (Sec. V-B): Nd(N') <= n_detail_eligible and N' - Nd(N') <= n_occupied. */
static int64_t nd_of(int64_t N, double frac) { return (int64_t)floor(frac * (double)N + 0.5); }

int64_t or_feasible_max(int64_t N, double frac, int64_t n_elig, int64_t n_occ)
{
    int64_t lo = 0, hi = N;          /* lo feasible, find the largest */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        int64_t nd = nd_of(mid, frac), nc = mid - nd;
        if (nd <= n_elig && nc <= n_occ) lo = mid; else hi = mid - 1;
    }
    return lo;
}

typedef struct { double key; int64_t idx; } dkey_t;
typedef struct { uint64_t key; int64_t idx; } ukey_t;

static int cmp_dkey(const void* a, const void* b)
{
    const dkey_t* x = (const dkey_t*)a; const dkey_t* y = (const dkey_t*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}
static int cmp_ukey(const void* a, const void* b)
{
    const ukey_t* x = (const ukey_t*)a; const ukey_t* y = (const ukey_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}
static int cmp_f32(const void* a, const void* b)
{
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}
static int cmp_f64(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Uniform double in (0,1) from two Philox words: 52 bits, (2m+1) 2^-53. */
static double unit_open(uint32_t x0, uint32_t x1)
{
    uint64_t m = (((uint64_t)x0 << 32) | x1) >> 12;
    return (double)(2 * m + 1) * 0x1p-53;
}

/* Efraimidis-Spirakis key for the detail draw at voxel v with weight g. */
double or_detail_key(uint64_t v, uint64_t seed, float g)
{
    uint32_t r[4];
    or_draw(v, 0u, seed, r);
    double u = unit_open(r[0], r[1]);
    return -log(u) / (double)g;
}

uint64_t or_coverage_key(uint64_t v, uint64_t seed)
{
    uint32_t r[4];
    or_draw(v, 1u, seed, r);
    return ((uint64_t)r[0] << 32) | r[1];
}

void or_jitter(uint64_t i, uint32_t group, uint64_t seed, float* u3)
{
    uint32_t r[4];
    or_draw(i, 2u + group, seed, r);
    for (int j = 0; j < 3; ++j) u3[j] = (float)(r[j] >> 8) * 0x1p-24f - 0.5f;
}

/* S1c: lower median over an evenly strided subsample (at most 4096) of the
 * mean distance from a seed to its 3 nearest seeds of the same group.
 * coords: voxel indices of the group's seeds, ascending. */
double or_group_spacing(const int64_t* vox, int64_t ng, const int dims[3], int64_t n_occ, int64_t N)
{
    if (ng < 2) return cbrt((double)(n_occ > 0 ? n_occ : 1) / (double)(N > 0 ? N : 1));
    int64_t nsub = ng < 4096 ? ng : 4096;
    int knn = ng - 1 < 3 ? (int)(ng - 1) : 3;
    double* vals = (double*)malloc(sizeof(double) * (size_t)nsub);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t j = 0; j < nsub; ++j) {
        int64_t i = (int64_t)(((__int128)j * ng) / nsub);
        int64_t vi = vox[i];
        int64_t xi = vi % dims[0], yi = (vi / dims[0]) % dims[1], zi = vi / ((int64_t)dims[0] * dims[1]);
        int64_t best[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
        for (int64_t o = 0; o < ng; ++o) {
            if (o == i) continue;
            int64_t vo = vox[o];
            int64_t dx = vo % dims[0] - xi, dy = (vo / dims[0]) % dims[1] - yi,
                    dz = vo / ((int64_t)dims[0] * dims[1]) - zi;
            int64_t d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best[2]) {
                if (d2 < best[1]) {
                    best[2] = best[1];
                    if (d2 < best[0]) { best[1] = best[0]; best[0] = d2; }
                    else best[1] = d2;
                } else best[2] = d2;
            }
        }
        double s = 0.0;
        for (int t = 0; t < knn; ++t) s += sqrt((double)best[t]);
        vals[j] = s / (double)knn;
    }
    qsort(vals, (size_t)nsub, sizeof(double), cmp_f64);
    double h = vals[(nsub - 1) / 2];
    free(vals);
    return h;
}

/* S1d + S1e for one seed at voxel v (|grad V| = gv there), index gi within
 * group grp: jitter (Eq. 4), 7^3 structure tensor, Jacobi, frame and
 * quaternion, scales s_t = sigma_g clamp(1 + gv / gbar, 1, 3), s_perp =
 * sigma_g with sigma_g = h_g / 2, all clamped to [0.3, max(dims) / 16],
 * a = trilinear V(mu), w_logit = logit(w0). */
static void assemble_seed(const float* V, const int dims[3], int64_t v, float gv, int64_t gi, int grp, uint64_t seed,
                          double h, double gbar, double wl, double* p)
{
    double smax_cap = (double)(dims[0] > dims[1] ? (dims[0] > dims[2] ? dims[0] : dims[2])
                                                 : (dims[1] > dims[2] ? dims[1] : dims[2])) / 16.0;
    double smin_cap = 0.3;
    int cx = (int)(v % dims[0]), cy = (int)((v / dims[0]) % dims[1]), cz = (int)(v / ((int64_t)dims[0] * dims[1]));
    float u[3];
    or_jitter((uint64_t)gi, (uint32_t)grp, seed, u);
    p[0] = cx + (double)u[0]; p[1] = cy + (double)u[1]; p[2] = cz + (double)u[2];
    double J6[6], ev[3], evec[9], R9[9], q[4];
    or_struct_tensor(V, dims, cx, cy, cz, J6);
    or_jacobi3(J6, ev, evec);
    canonical_frame(evec, R9);
    or_quat_from_R(R9, q);
    double sg = 0.5 * h;
    double ratio = gbar > 0.0 ? 1.0 + (double)gv / gbar : 1.0;
    if (ratio < 1.0) ratio = 1.0;
    if (ratio > 3.0) ratio = 3.0;
    double s[3] = {sg * ratio, sg, sg};
    for (int j = 0; j < 3; ++j) {
        if (s[j] > smax_cap) s[j] = smax_cap;
        if (s[j] < smin_cap) s[j] = smin_cap;
        p[3 + j] = log(s[j]);
    }
    p[6] = q[0]; p[7] = q[1]; p[8] = q[2]; p[9] = q[3];
    p[10] = or_trilinear(V, dims, p[0], p[1], p[2]);
    p[11] = wl;
}

typedef struct {
    int64_t n_occupied, n_eligible, n_detail, n_coverage, feasible_max;
    double gbar, h_detail, h_coverage;
} or_alloc_stats;

/* Full analytic allocation.  Returns 0 on success, 2 if the budget is
 * infeasible (stats->feasible_max set), 1 on error.  prm_out: [N][12] FP64;
 * vox_out (optional): [N] chosen voxel indices (detail first). */
int or_allocate(const float* V, const int dims[3], int64_t N, double detail_frac, float occ_thresh,
                double w0, uint64_t seed, double* prm_out, int64_t* vox_out, or_alloc_stats* st)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2];
    memset(st, 0, sizeof(*st));
    float* g = (float*)malloc(sizeof(float) * (size_t)M);
    if (!g) return 1;
    or_grad_mag32(V, dims, g);
    int64_t n_occ = 0, n_elig = 0;
    for (int64_t v = 0; v < M; ++v) {
        if (V[v] > occ_thresh) { ++n_occ; if (g[v] > 0.0f) ++n_elig; }
    }
    st->n_occupied = n_occ; st->n_eligible = n_elig;
    int64_t Nd = nd_of(N, detail_frac), Nc = N - Nd;
    st->n_detail = Nd; st->n_coverage = Nc;
    if (Nd > n_elig || Nc > n_occ) {
        st->feasible_max = or_feasible_max(N, detail_frac, n_elig, n_occ);
        free(g);
        return 2;
    }
    st->feasible_max = N;
    /* gbar: lower median of g over occupied voxels */
    float* go = (float*)malloc(sizeof(float) * (size_t)(n_occ > 0 ? n_occ : 1));
    int64_t t = 0;
    for (int64_t v = 0; v < M; ++v) if (V[v] > occ_thresh) go[t++] = g[v];
    qsort(go, (size_t)n_occ, sizeof(float), cmp_f32);
    double gbar = n_occ > 0 ? (double)go[(n_occ - 1) / 2] : 0.0;
    free(go);
    st->gbar = gbar;
    /* S1b: detail draw (weighted, distinct) and coverage draw (uniform, distinct) */
    dkey_t* dk = (dkey_t*)malloc(sizeof(dkey_t) * (size_t)(n_elig > 0 ? n_elig : 1));
    ukey_t* uk = (ukey_t*)malloc(sizeof(ukey_t) * (size_t)(n_occ > 0 ? n_occ : 1));
    int64_t a1 = 0, a2 = 0;
    for (int64_t v = 0; v < M; ++v) {
        if (!(V[v] > occ_thresh)) continue;
        uk[a2].key = or_coverage_key((uint64_t)v, seed); uk[a2].idx = v; ++a2;
        if (g[v] > 0.0f) { dk[a1].key = or_detail_key((uint64_t)v, seed, g[v]); dk[a1].idx = v; ++a1; }
    }
    qsort(dk, (size_t)a1, sizeof(dkey_t), cmp_dkey);
    qsort(uk, (size_t)a2, sizeof(ukey_t), cmp_ukey);
    int64_t* vd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Nd > 0 ? Nd : 1));
    int64_t* vc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Nc > 0 ? Nc : 1));
    for (int64_t i = 0; i < Nd; ++i) vd[i] = dk[i].idx;
    for (int64_t i = 0; i < Nc; ++i) vc[i] = uk[i].idx;
    free(dk); free(uk);
    qsort(vd, (size_t)Nd, sizeof(int64_t), cmp_i64);
    qsort(vc, (size_t)Nc, sizeof(int64_t), cmp_i64);
    /* S1c: group spacing */
    double hd = or_group_spacing(vd, Nd, dims, n_occ, N);
    double hc = or_group_spacing(vc, Nc, dims, n_occ, N);
    st->h_detail = hd; st->h_coverage = hc;
    double wl = log(w0 / (1.0 - w0));
    /* S1d + S1e per seed */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        int grp = i < Nd ? 0 : 1;
        int64_t gi = grp == 0 ? i : i - Nd;
        int64_t v = grp == 0 ? vd[gi] : vc[gi];
        if (vox_out) vox_out[i] = v;
        assemble_seed(V, dims, v, g[v], gi, grp, seed, grp == 0 ? hd : hc, gbar, wl, prm_out + 12 * i);
    }
    free(vd); free(vc); free(g);
    return 0;
}

/* S1d + S1e for caller-given seeds: voxel vox[i], index gi[i] within group
 * grp[i] (0 detail, 1 coverage), group spacings hd / hc, median gbar; the
 * same per-seed arithmetic as or_allocate.  out: [n][12]. */
void or_assemble_seeds(const float* V, const int dims[3], const int64_t* vox, const int64_t* gi, const int* grp,
                       int64_t n, uint64_t seed, double hd, double hc, double gbar, double w0, double* out)
{
    double wl = log(w0 / (1.0 - w0));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = vox[i];
        int x = (int)(v % dims[0]), y = (int)((v / dims[0]) % dims[1]), z = (int)(v / ((int64_t)dims[0] * dims[1]));
        assemble_seed(V, dims, v, gmag32_at(V, dims, x, y, z), gi[i], grp[i], seed, grp[i] == 0 ? hd : hc, gbar,
                      wl, out + 12 * i);
    }
}

/* Exhaustive census of the draws over the whole grid (Sec. III-E S1b), for
 * checking a draw made elsewhere at any size: out = {occupied voxels,
 * eligible voxels (occupied, |grad V| > 0), eligible voxels whose (detail
 * key, index) is at most (kd, kd_idx), occupied voxels whose (coverage key,
 * index) is at most (ku, ku_idx), occupied voxels with |grad V| < gbar,
 * occupied voxels with |grad V| <= gbar}. */
void or_draw_census(const float* V, const int dims[3], float occ_thresh, uint64_t seed, double kd, int64_t kd_idx,
                    uint64_t ku, int64_t ku_idx, float gbar, int64_t out[6])
{
    int64_t n_occ = 0, n_elig = 0, n_d = 0, n_u = 0, n_lt = 0, n_le = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_occ, n_elig, n_d, n_u, n_lt, n_le)
    for (int z = 0; z < dims[2]; ++z)
        for (int y = 0; y < dims[1]; ++y)
            for (int x = 0; x < dims[0]; ++x) {
                int64_t v = vidx(dims, x, y, z);
                if (!(V[v] > occ_thresh)) continue;
                ++n_occ;
                float g = gmag32_at(V, dims, x, y, z);
                n_lt += g < gbar;
                n_le += g <= gbar;
                uint64_t ukey = or_coverage_key((uint64_t)v, seed);
                n_u += ukey < ku || (ukey == ku && v <= ku_idx);
                if (g > 0.0f) {
                    ++n_elig;
                    double dkey = or_detail_key((uint64_t)v, seed, g);
                    n_d += dkey < kd || (dkey == kd && v <= kd_idx);
                }
            }
    out[0] = n_occ; out[1] = n_elig; out[2] = n_d; out[3] = n_u; out[4] = n_lt; out[5] = n_le;
}

/* Draw keys of listed voxels (for the census thresholds). */
void or_detail_keys(const int64_t* vox, const float* g, int64_t n, uint64_t seed, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = or_detail_key((uint64_t)vox[i], seed, g[i]);
}

void or_coverage_keys(const int64_t* vox, int64_t n, uint64_t seed, uint64_t* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = or_coverage_key((uint64_t)vox[i], seed);
}

/* Jitter of seeds 0..n-1 of one group: out [n][3]. */
void or_jitter_many(int64_t n, uint32_t group, uint64_t seed, float* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) or_jitter((uint64_t)i, group, seed, out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Stratified-sample refinement (Sec. III-F: each iteration fits the field  */
/* at a stratified set of jittered points; Table III: 3,072 per iteration,  */
/* 35 / 40 / 25 %).                                                          */
/* ------------------------------------------------------------------------ */
#define OR_SAMPLE_STREAM 4u

/* Voxel lists of the two value classes, ascending: high V > 0.4 and occupied
 * mid-range 0.02 < V <= 0.4 (float32 comparisons).  Either output may be
 * NULL to count only. */
void or_sample_classes(const float* V, const int dims[3], int64_t* hi, int64_t* n_hi, int64_t* mid, int64_t* n_mid)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2], a = 0, b = 0;
    for (int64_t v = 0; v < M; ++v) {
        if (V[v] > 0.4f) { if (hi) hi[a] = v; ++a; }
        else if (V[v] > 0.02f) { if (mid) mid[b] = v; ++b; }
    }
    *n_hi = a;
    *n_mid = b;
}

/* Per-class sample counts for S points: high floor(0.35 S + 1/2), mid
 * floor(0.40 S + 1/2), the rest uniform over the grid. */
void or_sample_split(int64_t S, int64_t out[3])
{
    out[0] = (int64_t)floor(0.35 * (double)S + 0.5);
    out[1] = (int64_t)floor(0.40 * (double)S + 0.5);
    out[2] = S - out[0] - out[1];
}

/* Sample j of iteration `iter`: Philox4x32-10 words x0..x3 of counter
 * (j, iter, 4, 'GVE1') under key seed.  Samples [0, n_hi) come from the
 * high class, the next n_mid from the mid class, the rest from all voxels;
 * a class with no voxel hands its samples to the uniform draw.  The voxel
 * is the floor(x0 * count / 2^32)-th of its class, the point p = c + u with
 * u_k = (x_{k+1} >> 8) 2^-24 - 1/2 (rounded once to float32), and the target
 * is the trilinear value V(p) (FP64, edge-clamped) rounded to float32. */
void or_draw_samples(const float* V, const int dims[3], const int64_t* hi, int64_t n_hi, const int64_t* mid,
                     int64_t n_mid, int64_t S, uint64_t seed, uint32_t iter, float* pts, float* vals, int64_t* vox)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2];
    int64_t split[3];
    or_sample_split(S, split);
    for (int64_t j = 0; j < S; ++j) {
        uint32_t r[4];
        or_draw(((uint64_t)iter << 32) | (uint64_t)(uint32_t)j, OR_SAMPLE_STREAM, seed, r);
        const int64_t* list = NULL;
        int64_t count = M;
        if (j < split[0] && n_hi > 0) { list = hi; count = n_hi; }
        else if (j >= split[0] && j < split[0] + split[1] && n_mid > 0) { list = mid; count = n_mid; }
        int64_t k = (int64_t)(((uint64_t)r[0] * (uint64_t)count) >> 32);
        int64_t v = list ? list[k] : k;
        int c[3] = {(int)(v % dims[0]), (int)((v / dims[0]) % dims[1]), (int)(v / ((int64_t)dims[0] * dims[1]))};
        for (int a = 0; a < 3; ++a) {
            float u = (float)(r[a + 1] >> 8) * 0x1p-24f - 0.5f;
            pts[3 * j + a] = (float)c[a] + u;
        }
        vals[j] = (float)or_trilinear(V, dims, (double)pts[3 * j], (double)pts[3 * j + 1], (double)pts[3 * j + 2]);
        if (vox) vox[j] = v;
    }
}

/* Keep exponent at a float32 point, by the same chain as at voxel centres. */
static float pred_t_at(const pred_t* P, float px, float py, float pz)
{
    float dx = px - P->mu[0];
    float dy = py - P->mu[1];
    float dz = pz - P->mu[2];
    float e = P->qxz2 * dz;
    float b = fmaf(P->qxy2, dy, e);
    float f = P->qyz2 * dz;
    float g = fmaf(P->qyy, dy, f);
    float hh = P->qzz * dz;
    float dzh = dz * hh;
    float c = fmaf(dy, g, dzh);
    float u = fmaf(P->qxx, dx, b);
    return fmaf(dx, u, c);
}

/* Eq. 3 at S points (every Gaussian against every point, kept by the float32
 * test) and the sampled value loss L = (1/S) sum_s 1[v_s > occ] (Vt_s - v_s)^2
 * with its gradient (grad may be NULL).  vt_out (optional) receives Vt_s. */
double or_sample_loss_grad(const double* prm, int64_t n, const float* pts, const float* vals, int64_t S, float k,
                           double rho0, double occ, double* grad, double* vt_out)
{
    act_t* A = (act_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(act_t));
    pred_t* P = (pred_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(pred_t));
    double* num = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
    double* den = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
    double* gn = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
    double* gd = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
    if (!A || !P || !num || !den || !gn || !gd) return NAN;
    const float T = pred_threshold(k);
    for (int64_t i = 0; i < n; ++i) {
        activate(prm + 12 * i, &A[i]);
        float p32[12];
        for (int j = 0; j < 12; ++j) p32[j] = (float)prm[12 * i + j];
        pred_coeffs(p32, &P[i]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; ++s) {
        const float* p = pts + 3 * s;
        double nu = 0.0, de = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (!A[i].valid || !P[i].valid) continue;
            if (!(pred_t_at(&P[i], p[0], p[1], p[2]) > T)) continue;
            double G = exp(-0.5 * maha2(&A[i], p[0], p[1], p[2]));
            nu += A[i].w * A[i].a * G;
            de += A[i].w * G;
        }
        num[s] = nu;
        den[s] = de;
    }
    double loss = 0.0;
    for (int64_t s = 0; s < S; ++s) {
        double vt = num[s] / (den[s] > rho0 ? den[s] : rho0);
        if (vt_out) vt_out[s] = vt;
        double r = vals[s] > (float)occ ? vt - (double)vals[s] : 0.0;
        loss += r * r;
        double up = 2.0 * r / (double)S;
        if (den[s] >= rho0) { gn[s] = up / den[s]; gd[s] = -vt * gn[s]; }
        else { gn[s] = up / rho0; gd[s] = 0.0; }
    }
    loss /= (double)S;
    if (grad) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double* out = grad + 12 * i;
            for (int j = 0; j < 12; ++j) out[j] = 0.0;
            if (!A[i].valid || !P[i].valid) continue;
            double Ag = 0, Bg = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0}};
            for (int64_t s = 0; s < S; ++s) {
                const float* p = pts + 3 * s;
                if (!(pred_t_at(&P[i], p[0], p[1], p[2]) > T)) continue;
                double d[3] = {p[0] - A[i].mu[0], p[1] - A[i].mu[1], p[2] - A[i].mu[2]};
                double Gv = exp(-0.5 * maha2(&A[i], p[0], p[1], p[2]));
                Ag += Gv * gn[s];
                Bg += Gv * gd[s];
                double c = A[i].w * (A[i].a * gn[s] + gd[s]);
                double h = -0.5 * c * Gv;
                for (int a2 = 0; a2 < 3; ++a2) {
                    S1[a2] += h * d[a2];
                    for (int b = 0; b < 3; ++b) S2[a2][b] += h * d[a2] * d[b];
                }
            }
            chain_rule(&A[i], prm + 12 * i, Ag, Bg, S1, S2, out);
        }
    }
    free(A); free(P); free(num); free(den); free(gn); free(gd);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* The full objective (Sec. III-F): the value term plus five regularisers    */
/* whose forms the paper gives in words only (the readings):                 */
/*   L_rho   = (1/S) sum_s 1[v_s > occ] (rho(p_s) - 1)^2, rho = sum w G      */
/*             (truncated like Eq. 3): density toward one over occupied      */
/*             space, from both sides;                                       */
/*   L_sm    = (1/S) sum_s (rho(p_s) - rho(p'_s))^2, p'_s a jittered partner */
/*             of p_s (pts[S + s]);                                          */
/*   L_anc   = (1/N) sum_i (a_i - V(mu_i))^2, V trilinear, gradient into a_i */
/*             only (the volume value is the anchor's target);               */
/*   L_aniso = (1/N) sum_i sum_{j<k} relu(|l_ij - l_ik| - ln r_max)^2,       */
/*             l = log-scales (elongation bounded at r_max : 1);             */
/*   L_cap   = (1/N) sum_i sum_j relu(l_ij - ln s_hi)^2                      */
/*             + relu(ln s_lo - l_ij)^2 (scales outside [s_lo, s_hi]).       */
/* ------------------------------------------------------------------------ */
#define OR_PARTNER_STREAM 5u

/* Partner of sample j of iteration iter: jitter u = (x >> 8) 2^-24 - 1/2 per
 * axis from Philox4x32-10 stream 5, counter (j, iter), scaled to
 * [-radius, radius) and the point clamped to [0, n - 1]; float32. */
void or_draw_partners(const float* pts, int64_t S, const int dims[3], uint64_t seed, uint32_t iter, float radius,
                      float* out)
{
    const float span = 2.0f * radius;
    for (int64_t j = 0; j < S; ++j) {
        uint32_t r[4];
        or_draw(((uint64_t)iter << 32) | (uint64_t)(uint32_t)j, OR_PARTNER_STREAM, seed, r);
        for (int a = 0; a < 3; ++a) {
            const float u = (float)(r[a] >> 8) * 0x1p-24f - 0.5f;
            float q = pts[3 * j + a] + u * span;
            const float hi = (float)(dims[a] - 1);
            q = q < 0.0f ? 0.0f : (q > hi ? hi : q);
            out[3 * j + a] = q;
        }
    }
}

/* lambda_sm at iteration t: geometric decay from l0 to l1 over `anneal`
 * iterations, then l1 (constant l0 when anneal <= 0 or l1 <= 0). */
double or_lambda_sm(double l0, double l1, int anneal, int t)
{
    if (anneal <= 0 || !(l1 > 0.0) || !(l0 > 0.0)) return l0;
    const double f = t < anneal ? (double)t / (double)anneal : 1.0;
    return l0 * pow(l1 / l0, f);
}

/* reg[8] = {l_rho, l_sm (this iteration's), l_anc, l_aniso, l_cap, r_max,
 * s_lo, s_hi}; pts holds S samples and, when smooth, their S partners after
 * them; field/dims give V for the anchor (may be NULL when l_anc = 0).
 * Returns L; terms[6] (optional) = {L_val, L_rho, L_sm, L_anc, L_aniso,
 * L_cap} unweighted; grad (optional) = dL/dprm. */
double or_sample_objective(const double* prm, int64_t n, const float* pts, const float* vals, int64_t S, int smooth,
                           const float* field, const int dims[3], const double* reg, float k, double rho0,
                           double occ, double* grad, double* terms)
{
    const int64_t P = smooth ? 2 * S : S;
    const double l_rho = reg[0], l_sm = reg[1], l_anc = reg[2], l_a = reg[3], l_s = reg[4];
    const double ln_r = log(reg[5]), ln_lo = log(reg[6]), ln_hi = log(reg[7]);
    act_t* A = (act_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(act_t));
    pred_t* Pc = (pred_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(pred_t));
    double* num = (double*)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    double* den = (double*)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    double* gn = (double*)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    double* gd = (double*)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    if (!A || !Pc || !num || !den || !gn || !gd) return NAN;
    const float T = pred_threshold(k);
    for (int64_t i = 0; i < n; ++i) {
        activate(prm + 12 * i, &A[i]);
        float p32[12];
        for (int j = 0; j < 12; ++j) p32[j] = (float)prm[12 * i + j];
        pred_coeffs(p32, &Pc[i]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < P; ++s) {
        const float* p = pts + 3 * s;
        double nu = 0.0, de = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (!A[i].valid || !Pc[i].valid) continue;
            if (!(pred_t_at(&Pc[i], p[0], p[1], p[2]) > T)) continue;
            double G = exp(-0.5 * maha2(&A[i], p[0], p[1], p[2]));
            nu += A[i].w * A[i].a * G;
            de += A[i].w * G;
        }
        num[s] = nu;
        den[s] = de;
    }
    /* point terms and the upstream gradient (dL/dnum, dL/dden) per point */
    double Lval = 0.0, Lrho = 0.0, Lsm = 0.0;
    for (int64_t s = 0; s < S; ++s) {
        const double vt = num[s] / (den[s] > rho0 ? den[s] : rho0);
        const int occd = vals[s] > (float)occ;
        const double r = occd ? vt - (double)vals[s] : 0.0;
        Lval += r * r;
        const double up = 2.0 * r / (double)S;
        if (den[s] >= rho0) { gn[s] = up / den[s]; gd[s] = -vt * gn[s]; }
        else { gn[s] = up / rho0; gd[s] = 0.0; }
        if (occd) {
            const double e = den[s] - 1.0;
            Lrho += e * e;
            gd[s] += l_rho * 2.0 * e / (double)S;
        }
        if (smooth) {
            const double e = den[s] - den[S + s];
            Lsm += e * e;
            gd[s] += l_sm * 2.0 * e / (double)S;
            gn[S + s] = 0.0;
            gd[S + s] = -l_sm * 2.0 * e / (double)S;
        }
    }
    Lval /= (double)S;
    Lrho /= (double)S;
    Lsm /= (double)S;
    if (grad) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double* out = grad + 12 * i;
            for (int j = 0; j < 12; ++j) out[j] = 0.0;
            if (!A[i].valid || !Pc[i].valid) continue;
            double Ag = 0, Bg = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0}};
            for (int64_t s = 0; s < P; ++s) {
                const float* p = pts + 3 * s;
                if (!(pred_t_at(&Pc[i], p[0], p[1], p[2]) > T)) continue;
                double d[3] = {p[0] - A[i].mu[0], p[1] - A[i].mu[1], p[2] - A[i].mu[2]};
                double Gv = exp(-0.5 * maha2(&A[i], p[0], p[1], p[2]));
                Ag += Gv * gn[s];
                Bg += Gv * gd[s];
                double c = A[i].w * (A[i].a * gn[s] + gd[s]);
                double h = -0.5 * c * Gv;
                for (int a2 = 0; a2 < 3; ++a2) {
                    S1[a2] += h * d[a2];
                    for (int b = 0; b < 3; ++b) S2[a2][b] += h * d[a2] * d[b];
                }
            }
            chain_rule(&A[i], prm + 12 * i, Ag, Bg, S1, S2, out);
        }
    }
    /* per-Gaussian terms */
    double Lanc = 0.0, Lan = 0.0, Lcap = 0.0;
    const double invN = n > 0 ? 1.0 / (double)n : 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!A[i].valid || !Pc[i].valid) continue;
        const double* q = prm + 12 * i;
        double* out = grad ? grad + 12 * i : NULL;
        if (l_anc != 0.0 && field) {
            const double r = q[10] - or_trilinear(field, dims, q[0], q[1], q[2]);
            Lanc += r * r;
            if (out) out[10] += l_anc * 2.0 * r * invN;
        }
        for (int j = 0; j < 3; ++j)
            for (int m = j + 1; m < 3; ++m) {
                const double dlt = q[3 + j] - q[3 + m];
                const double u = fabs(dlt) - ln_r;
                if (u > 0.0) {
                    Lan += u * u;
                    if (out) {
                        const double g = l_a * 2.0 * u * invN * (dlt > 0.0 ? 1.0 : -1.0);
                        out[3 + j] += g;
                        out[3 + m] -= g;
                    }
                }
            }
        for (int j = 0; j < 3; ++j) {
            const double u = q[3 + j] - ln_hi, w2 = ln_lo - q[3 + j];
            if (u > 0.0) { Lcap += u * u; if (out) out[3 + j] += l_s * 2.0 * u * invN; }
            if (w2 > 0.0) { Lcap += w2 * w2; if (out) out[3 + j] -= l_s * 2.0 * w2 * invN; }
        }
    }
    Lanc *= invN;
    Lan *= invN;
    Lcap *= invN;
    if (terms) {
        terms[0] = Lval; terms[1] = Lrho; terms[2] = Lsm; terms[3] = Lanc; terms[4] = Lan; terms[5] = Lcap;
    }
    free(A); free(Pc); free(num); free(den); free(gn); free(gd);
    return Lval + l_rho * Lrho + l_sm * Lsm + l_anc * Lanc + l_a * Lan + l_s * Lcap;
}

/* Regularised stratified-sample refinement.  regp[11] = {l_rho, l_sm0,
 * l_sm1, anneal_iters, l_anc, l_aniso, l_cap, r_max, s_lo, s_hi, radius}:
 * iteration t (index step0 + t) draws its samples, their partners when
 * l_sm0 > 0, takes L with l_sm = or_lambda_sm(l_sm0, l_sm1, anneal,
 * step0 + t), then one Adam step; losses[t] = L. */
int or_refine_sampled_reg(double* prm, int64_t n, const float* field, const int dims[3], int64_t S, uint64_t seed,
                          int step0, float k, double rho0, double occ, int iters, double lr, double b1, double b2,
                          double eps, const double* regp, double* losses)
{
    int64_t nh, nm;
    or_sample_classes(field, dims, NULL, &nh, NULL, &nm);
    int64_t* hi = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nh > 0 ? nh : 1));
    int64_t* mid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    float* pts = (float*)malloc(sizeof(float) * 6 * (size_t)S);
    float* vals = (float*)malloc(sizeof(float) * (size_t)S);
    double* g = (double*)malloc(sizeof(double) * 12 * (size_t)(n > 0 ? n : 1));
    double* m = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    double* v = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!hi || !mid || !pts || !vals || !g || !m || !v) return 1;
    or_sample_classes(field, dims, hi, &nh, mid, &nm);
    const int smooth = regp[1] > 0.0;
    for (int t = 0; t < iters; ++t) {
        const int step = step0 + t;
        or_draw_samples(field, dims, hi, nh, mid, nm, S, seed, (uint32_t)step, pts, vals, NULL);
        if (smooth) or_draw_partners(pts, S, dims, seed, (uint32_t)step, (float)regp[10], pts + 3 * S);
        const double reg[8] = {regp[0], or_lambda_sm(regp[1], regp[2], (int)regp[3], step), regp[4], regp[5],
                               regp[6], regp[7], regp[8], regp[9]};
        const double L = or_sample_objective(prm, n, pts, vals, S, smooth, field, dims, reg, k, rho0, occ, g, NULL);
        if (losses) losses[t] = L;
        or_adam(prm, m, v, g, 12 * n, step + 1, lr, b1, b2, eps);
    }
    free(hi); free(mid); free(pts); free(vals); free(g); free(m); free(v);
    return 0;
}

/* Stratified-sample refinement: iteration t draws its S points (iteration
 * index step0 + t), takes the sampled loss and gradient, then one Adam
 * step; losses[t] receives the sampled loss.  prm is updated in place. */
int or_refine_sampled(double* prm, int64_t n, const float* field, const int dims[3], int64_t S, uint64_t seed,
                      int step0, float k, double rho0, double occ, int iters, double lr, double b1, double b2,
                      double eps, double* losses)
{
    int64_t M = (int64_t)dims[0] * dims[1] * dims[2], nh, nm;
    or_sample_classes(field, dims, NULL, &nh, NULL, &nm);
    int64_t* hi = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nh > 0 ? nh : 1));
    int64_t* mid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    float* pts = (float*)malloc(sizeof(float) * 3 * (size_t)S);
    float* vals = (float*)malloc(sizeof(float) * (size_t)S);
    double* g = (double*)malloc(sizeof(double) * 12 * (size_t)(n > 0 ? n : 1));
    double* m = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    double* v = (double*)calloc(12 * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!hi || !mid || !pts || !vals || !g || !m || !v) return 1;
    or_sample_classes(field, dims, hi, &nh, mid, &nm);
    (void)M;
    for (int t = 0; t < iters; ++t) {
        or_draw_samples(field, dims, hi, nh, mid, nm, S, seed, (uint32_t)(step0 + t), pts, vals, NULL);
        double L = or_sample_loss_grad(prm, n, pts, vals, S, k, rho0, occ, g, NULL);
        if (losses) losses[t] = L;
        or_adam(prm, m, v, g, 12 * n, step0 + t + 1, lr, b1, b2, eps);
    }
    free(hi); free(mid); free(pts); free(vals); free(g); free(m); free(v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Mixture-field ray marching (Sec. III-A: rendering applies the transfer    */
/* function T = (c_T, alpha_T) to the value Eq. 3 returns at sample          */
/* positions and composites them along each ray; grad Vt is available for   */
/* shading at the sample).                                                   */
/*                                                                           */
/* Camera cam[13]: eye (3), right (3), up (3), forward (3), tan(fovy / 2),   */
/* in voxel coordinates (voxel centres at integers).  The ray through pixel  */
/* (i, j) (row 0 at the top) and its samples are set up in float32 in one    */
/* fixed order; values, shading and compositing are FP64.                    */
/* opt[12]: step, term (stop when the transmittance falls below; 0 = off),   */
/* ref_step (the spacing the table's opacities hold for), background RGB,    */
/* shade (0/1), ka, kd, ks, shininess, gfloor.                               */
/* ------------------------------------------------------------------------ */
int or_ray_setup(const float* cam, int W, int H, int i, int j, const int dims[3], float d[3], float* tmin,
                 float* tmax)
{
    const float* e = cam;
    const float *r = cam + 3, *u = cam + 6, *f = cam + 9;
    const float th = cam[12];
    const float aspect = (float)W / (float)H;
    const float sx = ((float)(2 * i + 1) / (float)W - 1.0f) * (th * aspect);
    const float sy = (1.0f - (float)(2 * j + 1) / (float)H) * th;
    float dd[3];
    for (int a = 0; a < 3; ++a) {
        const float t1 = f[a] + sx * r[a];
        dd[a] = t1 + sy * u[a];
    }
    const float n2a = dd[0] * dd[0] + dd[1] * dd[1];
    const float n2 = n2a + dd[2] * dd[2];
    if (!(n2 > 0.0f) || !isfinite(n2)) return 0;  /* degenerate camera: no ray */
    const float nrm = sqrtf(n2);
    for (int a = 0; a < 3; ++a) d[a] = dd[a] / nrm;
    float t0 = 0.0f, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const float lo = -0.5f, hi = (float)dims[a] - 0.5f;
        if (d[a] == 0.0f) {
            if (e[a] < lo || e[a] > hi) return 0;
            continue;
        }
        const float ta = (lo - e[a]) / d[a], tb = (hi - e[a]) / d[a];
        const float ta0 = ta < tb ? ta : tb, tb0 = ta < tb ? tb : ta;
        if (ta0 > t0) t0 = ta0;
        if (tb0 < t1) t1 = tb0;
    }
    *tmin = t0;
    *tmax = t1;
    return t0 < t1 && isfinite(t1);
}

typedef struct {
    act_t A;
    pred_t P;
    double half[3];  /* generous box: the float32 test keeps nothing outside */
    int ok;
} rg_t;

/* The oracle's own candidate index: cells of 16^3 voxels, each listing (in
 * index order) the Gaussians whose generous box reaches it.  It only skips
 * Gaussians the float32 test cannot keep; the sum over the rest is Eq. 3. */
typedef struct {
    int nc[3];
    int64_t* start;  /* [ncells + 1] */
    int64_t* ids;
} rindex_t;

static int rcell(double p, int nc)
{
    double f = floor((p + 0.5) / 16.0);
    if (f < 0) return 0;
    if (f > nc - 1) return nc - 1;
    return (int)f;
}

static int rindex_build(const rg_t* G, int64_t n, const int dims[3], rindex_t* X)
{
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        X->nc[a] = (dims[a] + 15) / 16;
        ncell *= X->nc[a];
    }
    X->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!X->start) return 1;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t* fill = NULL;
        if (pass == 1) {
            for (int64_t c = 0; c < ncell; ++c) X->start[c + 1] += X->start[c];
            X->ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(X->start[ncell] > 0 ? X->start[ncell] : 1));
            fill = (int64_t*)calloc((size_t)ncell, sizeof(int64_t));
            if (!X->ids || !fill) return 1;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (!G[i].ok) continue;
            int lo[3], hi[3], skip = 0;
            for (int a = 0; a < 3; ++a) {
                const double l = G[i].A.mu[a] - G[i].half[a], h = G[i].A.mu[a] + G[i].half[a];
                if (h < -0.5 || l > dims[a] - 0.5) skip = 1;
                lo[a] = rcell(l, X->nc[a]);
                hi[a] = rcell(h, X->nc[a]);
            }
            if (skip) continue;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const int64_t c = ((int64_t)z * X->nc[1] + y) * X->nc[0] + x;
                        if (pass == 0) X->start[c + 1]++;
                        else X->ids[X->start[c] + fill[c]++] = i;
                    }
        }
        free(fill);
    }
    return 0;
}

static rg_t* render_prepare(const double* prm, int64_t n, double k)
{
    rg_t* G = (rg_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(rg_t));
    if (!G) return NULL;
    for (int64_t i = 0; i < n; ++i) {
        activate(prm + 12 * i, &G[i].A);
        float p32[12];
        for (int q = 0; q < 12; ++q) p32[q] = (float)prm[12 * i + q];
        pred_coeffs(p32, &G[i].P);
        G[i].ok = G[i].A.valid && G[i].P.valid;
        for (int a = 0; a < 3; ++a) {
            double var = 0.0;
            for (int m = 0; m < 3; ++m) var += G[i].A.R[a][m] * G[i].A.R[a][m] * G[i].A.s[m] * G[i].A.s[m];
            G[i].half[a] = k * 1.01 * sqrt(var) + 0.5;
        }
    }
    return G;
}

/* Eq. 3 and its gradient at a float32 point; the float32 keep test decides
 * membership.  Normalised: Vt = N / max(D, rho0) and, where D > rho0, the
 * quotient rule (grad N D - N grad D) / D^2, else grad N / rho0. */
static void field_at(const rg_t* G, int64_t n, const rindex_t* X, float T, double rho0, int normalized,
                     const float p[3], double* v, double g[3], int64_t* kept)
{
    double N = 0.0, D = 0.0, gN[3] = {0, 0, 0}, gD[3] = {0, 0, 0};
    int64_t b = 0, e = n;
    if (X) {
        const int64_t c = ((int64_t)rcell(p[2], X->nc[2]) * X->nc[1] + rcell(p[1], X->nc[1])) * X->nc[0] +
                          rcell(p[0], X->nc[0]);
        b = X->start[c];
        e = X->start[c + 1];
    }
    for (int64_t ii = b; ii < e; ++ii) {
        const rg_t* q = &G[X ? X->ids[ii] : ii];
        if (!q->ok) continue;
        if (fabs((double)p[0] - q->A.mu[0]) > q->half[0] || fabs((double)p[1] - q->A.mu[1]) > q->half[1] ||
            fabs((double)p[2] - q->A.mu[2]) > q->half[2])
            continue;
        if (!(pred_t_at(&q->P, p[0], p[1], p[2]) > T)) continue;
        ++*kept;
        const double d[3] = {p[0] - q->A.mu[0], p[1] - q->A.mu[1], p[2] - q->A.mu[2]};
        double Cd[3], m = 0.0;
        for (int a = 0; a < 3; ++a) {
            Cd[a] = q->A.C[a][0] * d[0] + q->A.C[a][1] * d[1] + q->A.C[a][2] * d[2];
            m += d[a] * Cd[a];
        }
        const double Gv = exp(-0.5 * m);
        N += q->A.w * q->A.a * Gv;
        D += q->A.w * Gv;
        for (int a = 0; a < 3; ++a) {
            gN[a] -= q->A.w * q->A.a * Gv * Cd[a];
            gD[a] -= q->A.w * Gv * Cd[a];
        }
    }
    if (!normalized) {
        *v = N;
        for (int a = 0; a < 3; ++a) g[a] = gN[a];
    } else if (D > rho0) {
        *v = N / D;
        for (int a = 0; a < 3; ++a) g[a] = (gN[a] * D - N * gD[a]) / (D * D);
    } else {
        *v = N / rho0;
        for (int a = 0; a < 3; ++a) g[a] = gN[a] / rho0;
    }
}

int or_field_at(const double* prm, int64_t n, float k, double rho0, int normalized, const float* p, double* v,
                double* g, int64_t* kept)
{
    rg_t* G = render_prepare(prm, n, (double)k);
    if (!G) return 1;
    int64_t kk = 0;
    field_at(G, n, NULL, pred_threshold(k), rho0, normalized, p, v, g, &kk);
    if (kept) *kept = kk;
    free(G);
    return 0;
}

/* image: [H][W][4], or [npix][4] for the pixels pix[0..npix) (index j W + i)
 * when pix is given. */
int or_render(const double* prm, int64_t n, const int dims[3], float k, double rho0, int normalized,
              const float* cam, int W, int H, const float* opt, const float* tf, int tf_n, const int64_t* pix,
              int64_t npix, double* image, int64_t* kept_out, double* pixel_seconds)
{
    if (tf_n < 2 || W < 1 || H < 1 || !(opt[0] > 0.0f)) return 1;
    rg_t* G = render_prepare(prm, n, (double)k);
    if (!G) return 1;
    rindex_t X;
    memset(&X, 0, sizeof(X));
    if (rindex_build(G, n, dims, &X)) return 1;
    const int64_t np = pix ? npix : (int64_t)W * H;
    const float T = pred_threshold(k);
    const float step = opt[0];
    const double term = opt[1], ratio = (double)opt[0] / (double)opt[2];
    const int shade = opt[6] != 0.0f;
    const double ka = opt[7], kd = opt[8], ks = opt[9], shin = opt[10], gfloor = opt[11];
    int64_t kept_all = 0;
    struct timespec ts0, ts1;
    clock_gettime(CLOCK_MONOTONIC, &ts0);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : kept_all)
    for (int64_t q0 = 0; q0 < np; ++q0) {
        const int64_t px = pix ? pix[q0] : q0;
        const int i = (int)(px % W), j = (int)(px / W);
        float d[3], tmin, tmax;
        double Tr = 1.0, C[3] = {0.0, 0.0, 0.0};
        if (or_ray_setup(cam, W, H, i, j, dims, d, &tmin, &tmax)) {
            for (int64_t s = 0;; ++s) {
                const float t = tmin + ((float)s + 0.5f) * step;
                if (!(t < tmax)) break;
                float p[3];
                for (int a = 0; a < 3; ++a) p[a] = cam[a] + t * d[a];
                double v, g[3];
                int64_t kp = 0;
                field_at(G, n, &X, T, rho0, normalized, p, &v, g, &kp);
                kept_all += kp;
                /* transfer function: linear interpolation of the table on [0, 1] */
                const double u = (v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v)) * (double)(tf_n - 1);
                int i0 = (int)floor(u);
                if (i0 > tf_n - 2) i0 = tf_n - 2;
                const double fr = u - (double)i0;
                double c[4];
                for (int q = 0; q < 4; ++q) c[q] = (double)tf[4 * i0 + q] * (1.0 - fr) + (double)tf[4 * (i0 + 1) + q] * fr;
                const double a0 = c[3] < 0.0 ? 0.0 : (c[3] > 1.0 ? 1.0 : c[3]);
                const double as = 1.0 - pow(1.0 - a0, ratio);
                if (shade) {
                    const double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                    const double ndl = fabs(g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) / (gl > gfloor ? gl : gfloor);
                    const double sf = ka + kd * ndl, sp = ks * pow(ndl, shin);
                    for (int q = 0; q < 3; ++q) c[q] = c[q] * sf + sp;
                }
                for (int q = 0; q < 3; ++q) C[q] += Tr * as * c[q];
                Tr *= 1.0 - as;
                if (term > 0.0 && Tr < term) break;
            }
        }
        double* o = image + 4 * q0;
        for (int q = 0; q < 3; ++q) o[q] = C[q] + Tr * (double)opt[3 + q];
        o[3] = 1.0 - Tr;
    }
    clock_gettime(CLOCK_MONOTONIC, &ts1);
    if (pixel_seconds) *pixel_seconds = (double)(ts1.tv_sec - ts0.tv_sec) + 1e-9 * (double)(ts1.tv_nsec - ts0.tv_nsec);
    if (kept_out) *kept_out = kept_all;
    free(G);
    free(X.start);
    free(X.ids);
    return 0;
}
