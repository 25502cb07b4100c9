// chain.cuh -- the per-Gaussian chain rule and fused Adam step (device code
// shared by the chain-rule kernel and the batched persistent kernel).
//
// From the brick evaluator's sums -- A = sum G gn, H = sum h and the first
// and second moments S1', S2' of h = G (a gn + gd) over d = p - mu -- with
// S1 = -w S1'/2 and S2 = -w S2'/2 (the derivative of the loss with respect
// to the squared Mahalanobis distance being -w h / 2), to the gradient of the
// raw 12-float record of Eq. 2:
//   dL/da       = w A
//   dL/dw_logit = H w (1 - w)
//   dL/dmu      = -2 Sigma^-1 S1
//   dL/dlog s_j = -2 s_j^-2 (R^T S2 R)_jj
//   dL/dR       = 2 S2 R diag(s^-2)  -> dL/dq_hat -> dL/dq through q/|q|
// then either written out (gradient calls) or fed to Adam with bias
// correction (Kingma and Ba), in place on the record and its two moments.
// The accumulators are zeroed for the next iteration in the same pass when
// acc_zero is set.  An optional raw-record gradient (the per-Gaussian
// regularisers of the full objective) is added before the output or the
// Adam step.
#pragma once
#include "gve_int.cuh"

namespace gve {

// The chain rule and the optimiser step of Gaussian i.  acc and acc_zero
// may be the same buffer (read, then cleared): no __restrict__.
__device__ __forceinline__ void chain_one(const long long i, const float* acc, float* acc_zero, float* prims,
                                          float* grad, float* m, float* v, const AdamArgs& ad, const int do_adam,
                                          const float* extra)
{
    const float4* a4 = reinterpret_cast<const float4*>(acc) + 3 * i;
    const float4 c0 = a4[0], c1 = a4[1], c2 = a4[2];
    // the Adam moments are loaded with the sums, before any arithmetic, so
    // all of the record's loads are in flight at once
    float4 mv[6] = {};
    if (do_adam) {
        const float4* m4l = reinterpret_cast<const float4*>(m) + 3 * i;
        const float4* v4l = reinterpret_cast<const float4*>(v) + 3 * i;
        mv[0] = m4l[0]; mv[1] = m4l[1]; mv[2] = m4l[2];
        mv[3] = v4l[0]; mv[4] = v4l[1]; mv[5] = v4l[2];
    }
    if (acc_zero) {
        float4* z4 = reinterpret_cast<float4*>(acc_zero) + 3 * i;
        const float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
        z4[0] = zz; z4[1] = zz; z4[2] = zz;
    }
    float4* p4 = reinterpret_cast<float4*>(prims) + 3 * i;
    const float4 p0 = p4[0], p1 = p4[1], p2 = p4[2];
    float p[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
    float gr[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) gr[j] = 0.f;

    bool ok = true;
#pragma unroll
    for (int j = 0; j < 12; ++j) ok = ok && isfinite(p[j]);
    const float nq = sqrtf(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
    ok = ok && nq > 0.f && isfinite(nq);
    if (ok) {
        // accumulated: A = sum G gn, H = sum h, moments of h = G (a gn + gd)
        const float A = c0.x, H = c0.y;
        const float w = 1.f / (1.f + expf(-p[11]));
        const float hw = -0.5f * w;
        const float S1[3] = {hw * c0.z, hw * c0.w, hw * c1.x};
        const float sxx = hw * c1.y, syy = hw * c1.z, szz = hw * c1.w;
        const float sxy = hw * c2.x, sxz = hw * c2.y, syz = hw * c2.z;
        const float S2[3][3] = {{sxx, sxy, sxz}, {sxy, syy, syz}, {sxz, syz, szz}};
        float s[3], D[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { s[j] = expf(p[3 + j]); D[j] = 1.f / (s[j] * s[j]); }
        const float qw = p[6] / nq, qx = p[7] / nq, qy = p[8] / nq, qz = p[9] / nq;
        float R[3][3];
        R[0][0] = 1.f - 2.f * (qy * qy + qz * qz);
        R[0][1] = 2.f * (qx * qy - qw * qz);
        R[0][2] = 2.f * (qx * qz + qw * qy);
        R[1][0] = 2.f * (qx * qy + qw * qz);
        R[1][1] = 1.f - 2.f * (qx * qx + qz * qz);
        R[1][2] = 2.f * (qy * qz - qw * qx);
        R[2][0] = 2.f * (qx * qz - qw * qy);
        R[2][1] = 2.f * (qy * qz + qw * qx);
        R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
        // dL/dmu = -2 C S1, C = R D R^T
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float t = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float Cab = R[a][0] * R[b][0] * D[0] + R[a][1] * R[b][1] * D[1] + R[a][2] * R[b][2] * D[2];
                t += Cab * S1[b];
            }
            gr[a] = -2.f * t;
        }
        // S2 R
        float SR[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) SR[a][j] = S2[a][0] * R[0][j] + S2[a][1] * R[1][j] + S2[a][2] * R[2][j];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float Mjj = R[0][j] * SR[0][j] + R[1][j] * SR[1][j] + R[2][j] * SR[2][j];
            gr[3 + j] = -2.f * D[j] * Mjj;
        }
        float gR[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) gR[a][j] = 2.f * SR[a][j] * D[j];
        float gw = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        gy += gR[0][0] * (-4.f * qy); gz += gR[0][0] * (-4.f * qz);
        gw += gR[0][1] * (-2.f * qz); gx += gR[0][1] * (2.f * qy); gy += gR[0][1] * (2.f * qx); gz += gR[0][1] * (-2.f * qw);
        gw += gR[0][2] * (2.f * qy); gx += gR[0][2] * (2.f * qz); gy += gR[0][2] * (2.f * qw); gz += gR[0][2] * (2.f * qx);
        gw += gR[1][0] * (2.f * qz); gx += gR[1][0] * (2.f * qy); gy += gR[1][0] * (2.f * qx); gz += gR[1][0] * (2.f * qw);
        gx += gR[1][1] * (-4.f * qx); gz += gR[1][1] * (-4.f * qz);
        gw += gR[1][2] * (-2.f * qx); gx += gR[1][2] * (-2.f * qw); gy += gR[1][2] * (2.f * qz); gz += gR[1][2] * (2.f * qy);
        gw += gR[2][0] * (-2.f * qy); gx += gR[2][0] * (2.f * qz); gy += gR[2][0] * (-2.f * qw); gz += gR[2][0] * (2.f * qx);
        gw += gR[2][1] * (2.f * qx); gx += gR[2][1] * (2.f * qw); gy += gR[2][1] * (2.f * qz); gz += gR[2][1] * (2.f * qy);
        gx += gR[2][2] * (-4.f * qx); gy += gR[2][2] * (-4.f * qy);
        const float dot = gw * qw + gx * qx + gy * qy + gz * qz;
        gr[6] = (gw - qw * dot) / nq;
        gr[7] = (gx - qx * dot) / nq;
        gr[8] = (gy - qy * dot) / nq;
        gr[9] = (gz - qz * dot) / nq;
        gr[10] = w * A;
        gr[11] = H * w * (1.f - w);
    }
    if (extra) {
        const float4* x4 = reinterpret_cast<const float4*>(extra) + 3 * i;
        const float4 x0 = x4[0], x1 = x4[1], x2 = x4[2];
        const float xs[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
#pragma unroll
        for (int j = 0; j < 12; ++j) gr[j] += xs[j];
    }

    if (!do_adam) {
        float4* g4 = reinterpret_cast<float4*>(grad) + 3 * i;
        g4[0] = make_float4(gr[0], gr[1], gr[2], gr[3]);
        g4[1] = make_float4(gr[4], gr[5], gr[6], gr[7]);
        g4[2] = make_float4(gr[8], gr[9], gr[10], gr[11]);
        return;
    }
    float4* m4 = reinterpret_cast<float4*>(m) + 3 * i;
    float4* v4 = reinterpret_cast<float4*>(v) + 3 * i;
    float mm[12], vv[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 a = mv[k], b = mv[3 + k];
        mm[4 * k] = a.x; mm[4 * k + 1] = a.y; mm[4 * k + 2] = a.z; mm[4 * k + 3] = a.w;
        vv[4 * k] = b.x; vv[4 * k + 1] = b.y; vv[4 * k + 2] = b.z; vv[4 * k + 3] = b.w;
    }
    const float bc1 = ad.bc_dev ? ad.bc_dev[0] : ad.bc1;
    const float bc2 = ad.bc_dev ? ad.bc_dev[1] : ad.bc2;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        mm[j] = ad.b1 * mm[j] + (1.f - ad.b1) * gr[j];
        vv[j] = ad.b2 * vv[j] + (1.f - ad.b2) * gr[j] * gr[j];
        const float mh = mm[j] / bc1, vh = vv[j] / bc2;
        p[j] -= ad.lr * mh / (sqrtf(vh) + ad.eps);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m4[k] = make_float4(mm[4 * k], mm[4 * k + 1], mm[4 * k + 2], mm[4 * k + 3]);
        v4[k] = make_float4(vv[4 * k], vv[4 * k + 1], vv[4 * k + 2], vv[4 * k + 3]);
        p4[k] = make_float4(p[4 * k], p[4 * k + 1], p[4 * k + 2], p[4 * k + 3]);
    }
}

}  // namespace gve
