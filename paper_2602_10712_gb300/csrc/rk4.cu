// rk4.cu -- orbit and attitude integration of Sec. 3.4 (Eq. "ODE") with
// fourth-order Runge-Kutta in FP64 and its discrete adjoint.
//
// State z (13): r, v (inertial), unit quaternion q = (q0,q1,q2,q3) taking
// body vectors to inertial, body rate w.
//   r' = v
//   v' = R(q) F / m + gravity(r)           (two-body + J2)
//   q' = 1/2 q (x) (0, w)
//   w' = I^-1 (tau - w x I w)              (I diagonal)
// (F, tau) = P (std * y + mean) with y the force model evaluated at the
// body-frame sun direction wbar = R(q)^T e_sun and the design theta:
//   proxy:      y = MLP(scale * (wbar, theta) + offset)   (FP32, Sec. 3.3)
//   cannonball: y = (-theta_0 wbar, 0, 0, 0)
//   none:       y = 0
//
// One CTA of 256 threads integrates one trajectory.  The MLP is evaluated
// by all threads (weights transposed for coalesced reads); the FP64 state
// algebra runs on a few threads.  Adjoint: reverse sweep over the discrete
// RK4 map with checkpoints every C steps; a segment is recomputed into
// shared memory and swept backwards.  The vector-Jacobian products of the
// dynamics use forward-mode dual numbers over the same templated dyn():
// 13 passes seeded on z, 6 on y and 4 on q (for wbar(q)) run on 23 threads
// at once; the MLP's input gradient is back-propagated by all threads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "srp_internal.h"

namespace srp {

struct OrbitDev {
    double mu, j2, re, mass, I[3], P, sun[3], dt;
    int n_steps, ckpt, model, n_theta;
    int eclipse;                          // cylinder shadow switches SRP off
    double gm3[2], pos3[2][3];            // point masses at fixed positions (GM 0 = off)
    float in_scale[19], in_offset[19], out_mean[6], out_std[6];
    // proxy weights (FP32): W_l [out][in], Wt_l [in][out], b_l
    const float* W[5];
    const float* Wt[5];
    const float* b[5];
};

constexpr int kMaxCkptSeg = 64;

// ---- dual numbers ------------------------------------------------------------
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d = 0.0) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
    const double s = sqrt(a.v);
    return {s, a.d / (2.0 * s)};
}
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }

template <class S>
__device__ __forceinline__ S cst(double v) { return S(v); }
template <>
__device__ __forceinline__ Dual cst<Dual>(double v) { return Dual{v, 0.0}; }

// body-frame sun direction wbar = R(q)^T e
template <class S>
__device__ void sun_body(const S* q, const double* e, S* wb) {
    const S q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    const S two = cst<S>(2.0);
    const S R00 = q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, R01 = two * (q1 * q2 - q0 * q3), R02 = two * (q1 * q3 + q0 * q2);
    const S R10 = two * (q1 * q2 + q0 * q3), R11 = q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, R12 = two * (q2 * q3 - q0 * q1);
    const S R20 = two * (q1 * q3 - q0 * q2), R21 = two * (q2 * q3 + q0 * q1), R22 = q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3;
    wb[0] = e[0] * R00 + e[1] * R10 + e[2] * R20;
    wb[1] = e[0] * R01 + e[1] * R11 + e[2] * R21;
    wb[2] = e[0] * R02 + e[1] * R12 + e[2] * R22;
}

// the dynamics k = f(z, y) for a given force-model output y (6)
template <class S>
__device__ void dyn(const OrbitDev& o, const S* z, const S* y, S* k) {
    const S x = z[0], yy = z[1], zz = z[2];
    // cylinder eclipse (decided on the values; piecewise constant in r)
    double nu = 1.0;
    if (o.eclipse) {
        const double rx = val(x), ry = val(yy), rz = val(zz);
        const double pr = rx * o.sun[0] + ry * o.sun[1] + rz * o.sun[2];
        if (pr < 0.0 && (rx * rx + ry * ry + rz * rz - pr * pr) < o.re * o.re) nu = 0.0;
    }
    const S q0 = z[6], q1 = z[7], q2 = z[8], q3 = z[9];
    const S w0 = z[10], w1 = z[11], w2 = z[12];
    const S two = cst<S>(2.0);
    // rotation body -> inertial
    const S R00 = q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, R01 = two * (q1 * q2 - q0 * q3), R02 = two * (q1 * q3 + q0 * q2);
    const S R10 = two * (q1 * q2 + q0 * q3), R11 = q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, R12 = two * (q2 * q3 - q0 * q1);
    const S R20 = two * (q1 * q3 - q0 * q2), R21 = two * (q2 * q3 + q0 * q1), R22 = q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3;
    S F[3], T[3];
    for (int j = 0; j < 3; ++j) {
        F[j] = (nu * o.P) * (cst<S>((double)o.out_std[j]) * y[j] + cst<S>((double)o.out_mean[j]));
        T[j] = (nu * o.P) * (cst<S>((double)o.out_std[3 + j]) * y[3 + j] + cst<S>((double)o.out_mean[3 + j]));
    }
    // gravity: two-body + J2
    const S r2 = x * x + yy * yy + zz * zz;
    const S rn = dsqrt(r2);
    const S c1 = cst<S>(-o.mu) / (rn * r2);
    const S kj = cst<S>(-1.5 * o.j2 * o.mu * o.re * o.re) / (r2 * r2 * rn);
    const S f5 = cst<S>(5.0) * zz * zz / r2;
    const S one = cst<S>(1.0), three = cst<S>(3.0);
    const double im = 1.0 / o.mass;
    k[0] = z[3]; k[1] = z[4]; k[2] = z[5];
    k[3] = im * (R00 * F[0] + R01 * F[1] + R02 * F[2]) + c1 * x + kj * x * (one - f5);
    k[4] = im * (R10 * F[0] + R11 * F[1] + R12 * F[2]) + c1 * yy + kj * yy * (one - f5);
    k[5] = im * (R20 * F[0] + R21 * F[1] + R22 * F[2]) + c1 * zz + kj * zz * (three - f5);
    // point masses at fixed positions: GM [(s - r)/|s - r|^3 - s/|s|^3]
    for (int b = 0; b < 2; ++b) {
        if (o.gm3[b] == 0.0) continue;
        const double* sp = o.pos3[b];
        const S dx = cst<S>(sp[0]) - x, dy = cst<S>(sp[1]) - yy, dz = cst<S>(sp[2]) - zz;
        const S d2 = dx * dx + dy * dy + dz * dz;
        const S g = cst<S>(o.gm3[b]) / (d2 * dsqrt(d2));
        const double s2 = sp[0] * sp[0] + sp[1] * sp[1] + sp[2] * sp[2];
        const double gs = o.gm3[b] / (s2 * std::sqrt(s2));
        k[3] = k[3] + g * dx - cst<S>(gs * sp[0]);
        k[4] = k[4] + g * dy - cst<S>(gs * sp[1]);
        k[5] = k[5] + g * dz - cst<S>(gs * sp[2]);
    }
    const S half = cst<S>(0.5);
    k[6] = half * (-(q1 * w0) - q2 * w1 - q3 * w2);
    k[7] = half * (q0 * w0 + q2 * w2 - q3 * w1);
    k[8] = half * (q0 * w1 + q3 * w0 - q1 * w2);
    k[9] = half * (q0 * w2 + q1 * w1 - q2 * w0);
    const S Iw0 = o.I[0] * w0, Iw1 = o.I[1] * w1, Iw2 = o.I[2] * w2;
    k[10] = (1.0 / o.I[0]) * (T[0] - (w1 * Iw2 - w2 * Iw1));
    k[11] = (1.0 / o.I[1]) * (T[1] - (w2 * Iw0 - w0 * Iw2));
    k[12] = (1.0 / o.I[2]) * (T[2] - (w0 * Iw1 - w1 * Iw0));
}

// ---- shared memory of one trajectory CTA --------------------------------------
struct OrbitSmem {
    double z[13], u[13], k[4][13], acc[13];
    double lam[13], zbar[13], kbar[4][13], vj_z[13], vj_th[16];
    double seg[kMaxCkptSeg + 1][13];
    double dpass[23];
    double wb[3];
    float x[32];         // model input
    float zpre[4][256];  // hidden pre-activations
    float h[2][256];
    float y[8], ybar[8];
    float g[2][256];     // back-propagated gradients
    float xbar[32];
    double theta[16];
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// y = model(wbar, theta); keeps the hidden pre-activations for the VJP.
__device__ void model_fwd(const OrbitDev& o, OrbitSmem& s) {
    const int t = threadIdx.x;
    if (o.model != 2) {  // none / cannonball: on thread 0
        if (t == 0) {
            for (int j = 0; j < 6; ++j) s.y[j] = 0.0f;
            if (o.model == 1)
                for (int j = 0; j < 3; ++j) s.y[j] = (float)(-s.theta[0] * s.wb[j]);
        }
        __syncthreads();
        return;
    }
    if (t < 19) {
        const double xv = t < 3 ? s.wb[t] : s.theta[t - 3];
        s.x[t] = (float)(o.in_scale[t] * xv + o.in_offset[t]);
    }
    __syncthreads();
    {  // layer 0: 19 -> 256
        float a = o.b[0][t];
        for (int i = 0; i < 19; ++i) a = fmaf(o.Wt[0][i * 256 + t], s.x[i], a);
        s.zpre[0][t] = a;
        s.h[0][t] = silu_f(a);
    }
    __syncthreads();
    for (int l = 1; l < 4; ++l) {
        const float* hin = s.h[(l - 1) & 1];
        const float* Wt = o.Wt[l];
        // 32 weight loads in flight per thread and four partial sums: the
        // loop is bound by the latency of the weight stream from L2
        float a0 = o.b[l][t], a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        for (int i = 0; i < 256; i += 32) {
            float w[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) w[u] = __ldg(Wt + (i + u) * 256 + t);
#pragma unroll
            for (int u = 0; u < 32; u += 4) {
                a0 = fmaf(w[u], hin[i + u], a0);
                a1 = fmaf(w[u + 1], hin[i + u + 1], a1);
                a2 = fmaf(w[u + 2], hin[i + u + 2], a2);
                a3 = fmaf(w[u + 3], hin[i + u + 3], a3);
            }
        }
        const float a = (a0 + a1) + (a2 + a3);
        s.zpre[l][t] = a;
        s.h[l & 1][t] = silu_f(a);
        __syncthreads();
    }
    {  // layer 4: 256 -> 6, warps 0..5 reduce one output each
        const int w = t >> 5, lane = t & 31;
        if (w < 6) {
            const float* hin = s.h[1];
            float a = 0.0f;
            for (int i = lane; i < 256; i += 32) a = fmaf(o.W[4][w * 256 + i], hin[i], a);
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) s.y[w] = a + o.b[4][w];
        }
    }
    __syncthreads();
}

// xbar = (d model / d x)^T ybar, then (wbar_bar, theta_bar) in s.xbar[0..2], [3..].
__device__ void model_vjp(const OrbitDev& o, OrbitSmem& s) {
    const int t = threadIdx.x;
    if (o.model != 2) {
        if (t == 0) {
            for (int j = 0; j < 19; ++j) s.xbar[j] = 0.0f;
            if (o.model == 1) {  // y[0:3] = -theta0 wbar
                float tb = 0.0f;
                for (int j = 0; j < 3; ++j) {
                    s.xbar[j] = (float)(-s.theta[0]) * s.ybar[j];
                    tb += (float)(-s.wb[j]) * s.ybar[j];
                }
                s.xbar[3] = tb;
            }
        }
        __syncthreads();
        return;
    }
    {  // dh4[i] = sum_o W4[o][i] ybar[o];  dz3 = dh4 * silu'(z3)
        float a = 0.0f;
        for (int oo = 0; oo < 6; ++oo) a = fmaf(o.W[4][oo * 256 + t], s.ybar[oo], a);
        s.g[0][t] = a * dsilu_f(s.zpre[3][t]);
    }
    __syncthreads();
    int cur = 0;
    for (int l = 3; l >= 1; --l) {  // dh_l[i] = sum_o W_l[o][i] dz_l[o]; dz_{l-1} = dh_l * silu'(z_{l-1})
        const float* gin = s.g[cur];
        const float* W = o.W[l];
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        for (int oo = 0; oo < 256; oo += 32) {
            float w[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) w[u] = __ldg(W + (oo + u) * 256 + t);
#pragma unroll
            for (int u = 0; u < 32; u += 4) {
                a0 = fmaf(w[u], gin[oo + u], a0);
                a1 = fmaf(w[u + 1], gin[oo + u + 1], a1);
                a2 = fmaf(w[u + 2], gin[oo + u + 2], a2);
                a3 = fmaf(w[u + 3], gin[oo + u + 3], a3);
            }
        }
        const float a = (a0 + a1) + (a2 + a3);
        s.g[cur ^ 1][t] = a * dsilu_f(s.zpre[l - 1][t]);
        __syncthreads();
        cur ^= 1;
    }
    {  // dx[i] = sum_o W0[o][i] dz0[o], i < 19: warps reduce
        const int w = t >> 5, lane = t & 31;
        for (int i = w; i < 19; i += 8) {
            float a = 0.0f;
            for (int oo = lane; oo < 256; oo += 32) a = fmaf(o.W[0][oo * 19 + i], s.g[cur][oo], a);
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) s.xbar[i] = a * o.in_scale[i];
        }
    }
    __syncthreads();
}

// k_out = f(u) (u in s.u); leaves wbar and the model state in smem.
__device__ void feval(const OrbitDev& o, OrbitSmem& s, double* kout) {
    if (threadIdx.x == 0) sun_body<double>(s.u + 6, o.sun, s.wb);
    __syncthreads();
    model_fwd(o, s);
    if (threadIdx.x == 0) {
        double yd[6];
        for (int j = 0; j < 6; ++j) yd[j] = (double)s.y[j];
        dyn<double>(o, s.u, yd, kout);
    }
    __syncthreads();
}

// VJP of f at u = s.u with cotangent lam_k: vj_z (13) and vj_th (n_theta).
__device__ void fvjp(const OrbitDev& o, OrbitSmem& s, const double* lam_k) {
    const int t = threadIdx.x;
    if (t == 0) sun_body<double>(s.u + 6, o.sun, s.wb);
    __syncthreads();
    model_fwd(o, s);
    // dual passes: 0..12 seed z_i, 13..18 seed y_j, 19..22 seed q_j in wbar(q)
    if (t < 23) {
        if (t < 19) {
            Dual z[13], y[6], k[13];
            for (int j = 0; j < 13; ++j) z[j] = mk(s.u[j], t == j ? 1.0 : 0.0);
            for (int j = 0; j < 6; ++j) y[j] = mk((double)s.y[j], t == 13 + j ? 1.0 : 0.0);
            dyn<Dual>(o, z, y, k);
            double acc = 0.0;
            for (int j = 0; j < 13; ++j) acc += lam_k[j] * k[j].d;
            s.dpass[t] = acc;
        }
    }
    __syncthreads();
    if (t < 6) s.ybar[t] = (float)s.dpass[13 + t];
    __syncthreads();
    model_vjp(o, s);
    // wbar(q) back to q: pass t = 19..22 seeds q_{t-19}
    if (t >= 19 && t < 23) {
        Dual q[4], wb[3];
        for (int j = 0; j < 4; ++j) q[j] = mk(s.u[6 + j], (t - 19) == j ? 1.0 : 0.0);
        sun_body<Dual>(q, o.sun, wb);
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += (double)s.xbar[j] * wb[j].d;
        s.dpass[t] = acc;
    }
    __syncthreads();
    if (t < 13) s.vj_z[t] = s.dpass[t] + (t >= 6 && t < 10 ? s.dpass[19 + t - 6] : 0.0);
    if (t < o.n_theta) s.vj_th[t] = (double)s.xbar[3 + t];
    __syncthreads();
}

// one RK4 step z -> z (in place), using s.u and s.k
__device__ void rk4_step(const OrbitDev& o, OrbitSmem& s, double* z) {
    const int t = threadIdx.x;
    const double h = o.dt;
    if (t < 13) s.u[t] = z[t];
    __syncthreads();
    feval(o, s, s.k[0]);
    if (t < 13) s.u[t] = z[t] + 0.5 * h * s.k[0][t];
    __syncthreads();
    feval(o, s, s.k[1]);
    if (t < 13) s.u[t] = z[t] + 0.5 * h * s.k[1][t];
    __syncthreads();
    feval(o, s, s.k[2]);
    if (t < 13) s.u[t] = z[t] + h * s.k[2][t];
    __syncthreads();
    feval(o, s, s.k[3]);
    if (t < 13) z[t] = z[t] + (h / 6.0) * (s.k[0][t] + 2.0 * s.k[1][t] + 2.0 * s.k[2][t] + s.k[3][t]);
    __syncthreads();
}

__global__ void __launch_bounds__(256) rk4_forward_kernel(const OrbitDev o, const double* __restrict__ z0,
                                                          const double* __restrict__ theta, double* zN, double* traj,
                                                          double* ckpt, int n_ck) {
    __shared__ OrbitSmem s;
    const int tr = blockIdx.x, t = threadIdx.x;
    if (t < 13) s.z[t] = z0[(size_t)tr * 13 + t];
    if (t < o.n_theta) s.theta[t] = theta[(size_t)tr * o.n_theta + t];
    __syncthreads();
    for (int n = 0; n < o.n_steps; ++n) {
        if (t < 13) {
            if (traj) traj[((size_t)tr * (o.n_steps + 1) + n) * 13 + t] = s.z[t];
            if (ckpt && n % o.ckpt == 0) ckpt[((size_t)tr * n_ck + n / o.ckpt) * 13 + t] = s.z[t];
        }
        rk4_step(o, s, s.z);
    }
    if (t < 13) {
        if (traj) traj[((size_t)tr * (o.n_steps + 1) + o.n_steps) * 13 + t] = s.z[t];
        zN[(size_t)tr * 13 + t] = s.z[t];
    }
}

__global__ void __launch_bounds__(256) rk4_adjoint_kernel(const OrbitDev o, const double* __restrict__ theta,
                                                          const double* __restrict__ ckpt, int n_ck,
                                                          const double* __restrict__ lamN, double* dth, double* dz0) {
    __shared__ OrbitSmem s;
    __shared__ double thbar[16];
    const int tr = blockIdx.x, t = threadIdx.x;
    const double h = o.dt;
    if (t < 13) s.lam[t] = lamN[(size_t)tr * 13 + t];
    if (t < 16) thbar[t] = 0.0;
    if (t < o.n_theta) s.theta[t] = theta[(size_t)tr * o.n_theta + t];
    __syncthreads();
    for (int sgi = n_ck - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * o.ckpt;
        const int n1 = min(o.n_steps, n0 + o.ckpt);
        // recompute the segment's states
        if (t < 13) { s.seg[0][t] = ckpt[((size_t)tr * n_ck + sgi) * 13 + t]; s.z[t] = s.seg[0][t]; }
        __syncthreads();
        for (int n = n0; n < n1 - 1; ++n) {
            rk4_step(o, s, s.z);
            if (t < 13) s.seg[n - n0 + 1][t] = s.z[t];
            __syncthreads();
        }
        // reverse sweep over the segment
        for (int n = n1 - 1; n >= n0; --n) {
            double* zn = s.seg[n - n0];
            // stage inputs and slopes
            if (t < 13) s.u[t] = zn[t];
            __syncthreads();
            feval(o, s, s.k[0]);
            if (t < 13) s.u[t] = zn[t] + 0.5 * h * s.k[0][t];
            __syncthreads();
            feval(o, s, s.k[1]);
            if (t < 13) s.u[t] = zn[t] + 0.5 * h * s.k[1][t];
            __syncthreads();
            feval(o, s, s.k[2]);
            if (t < 13) {
                s.kbar[3][t] = h / 6.0 * s.lam[t];
                s.kbar[2][t] = h / 3.0 * s.lam[t];
                s.kbar[1][t] = h / 3.0 * s.lam[t];
                s.kbar[0][t] = h / 6.0 * s.lam[t];
                s.zbar[t] = s.lam[t];
            }
            __syncthreads();
            // stage 4: u4 = z + h k3
            if (t < 13) s.u[t] = zn[t] + h * s.k[2][t];
            __syncthreads();
            fvjp(o, s, s.kbar[3]);
            if (t < 13) { s.zbar[t] += s.vj_z[t]; s.kbar[2][t] += h * s.vj_z[t]; }
            if (t < o.n_theta) thbar[t] += s.vj_th[t];
            // stage 3: u3 = z + h/2 k2
            if (t < 13) s.u[t] = zn[t] + 0.5 * h * s.k[1][t];
            __syncthreads();
            fvjp(o, s, s.kbar[2]);
            if (t < 13) { s.zbar[t] += s.vj_z[t]; s.kbar[1][t] += 0.5 * h * s.vj_z[t]; }
            if (t < o.n_theta) thbar[t] += s.vj_th[t];
            // stage 2: u2 = z + h/2 k1
            if (t < 13) s.u[t] = zn[t] + 0.5 * h * s.k[0][t];
            __syncthreads();
            fvjp(o, s, s.kbar[1]);
            if (t < 13) { s.zbar[t] += s.vj_z[t]; s.kbar[0][t] += 0.5 * h * s.vj_z[t]; }
            if (t < o.n_theta) thbar[t] += s.vj_th[t];
            // stage 1: u1 = z
            if (t < 13) s.u[t] = zn[t];
            __syncthreads();
            fvjp(o, s, s.kbar[0]);
            if (t < 13) { s.zbar[t] += s.vj_z[t]; s.lam[t] = s.zbar[t]; }
            if (t < o.n_theta) thbar[t] += s.vj_th[t];
            __syncthreads();
        }
    }
    if (t < 13 && dz0) dz0[(size_t)tr * 13 + t] = s.lam[t];
    if (t < o.n_theta && dth) dth[(size_t)tr * o.n_theta + t] = thbar[t];
}

// Wt_l[i][o] = W_l[o][i]
__global__ void transpose_kernel(const float* __restrict__ W, float* __restrict__ Wt, int out, int in) {
    const int64_t n = (int64_t)out * in;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int oo = (int)(e / in), i = (int)(e % in);
        Wt[(int64_t)i * out + oo] = W[e];
    }
}

int64_t mlp_param_count();
void set_last_error(const std::string& msg);
cudaStream_t ctx_stream(srp_ctx* c);
int ctx_device(srp_ctx* c);
const float* mlp_params_ptr(const srp_mlp* m);

}  // namespace srp

using namespace srp;

namespace {
int ofail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}
#define OCU(call, where)                                                                                   \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return ofail(SRP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)
}  // namespace

extern "C" void srp_orbit_opts_default(srp_orbit_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mu = 3.986004418e14; o->j2 = 1.08263e-3; o->re = 6378137.0;
    o->mass = 1000.0; o->inertia[0] = 500.0; o->inertia[1] = 400.0; o->inertia[2] = 300.0;
    o->pressure = 1361.0 / 299792458.0;
    o->sun[0] = 1.0;
    o->dt = 60.0; o->n_steps = 1440; o->ckpt_every = 0; o->model = SRP_FM_NONE; o->n_theta = 1;
    for (int j = 0; j < 19; ++j) o->in_scale[j] = 1.0f;
    for (int j = 0; j < 6; ++j) o->out_std[j] = 1.0f;
    o->eclipse = 0;
    o->gm_sun = 0.0; o->sun_dist = 1.495978707e11;
    o->gm_moon = 0.0;
}

extern "C" int srp_integrate(srp_ctx* c, const srp_orbit_opts* oo, const srp_mlp* proxy, int n_traj,
                             const double* z0, const double* theta, double* zN, double* traj,
                             const double* dL_dzN, double* dL_dtheta, double* dL_dz0, int mem) {
    if (!c || !oo) return ofail(SRP_EINVAL, "srp_integrate: NULL ctx/opts");
    if (n_traj < 0) return ofail(SRP_EINVAL, "srp_integrate: negative n_traj");
    if (oo->n_steps < 0 || !(oo->dt > 0.0)) return ofail(SRP_EINVAL, "srp_integrate: need n_steps >= 0, dt > 0");
    if (oo->model < SRP_FM_NONE || oo->model > SRP_FM_PROXY) return ofail(SRP_EINVAL, "srp_integrate: bad model");
    if (oo->n_theta < 1 || oo->n_theta > 16) return ofail(SRP_EINVAL, "srp_integrate: n_theta must be 1..16");
    if (oo->model == SRP_FM_PROXY && (!proxy || oo->n_theta != 16))
        return ofail(SRP_EINVAL, "srp_integrate: the proxy model needs an srp_mlp and n_theta = 16");
    if (!(oo->mass > 0) || !(oo->inertia[0] > 0) || !(oo->inertia[1] > 0) || !(oo->inertia[2] > 0))
        return ofail(SRP_EINVAL, "srp_integrate: mass and inertia must be positive");
    if (oo->eclipse != 0 && oo->eclipse != 1) return ofail(SRP_EINVAL, "srp_integrate: eclipse must be 0 or 1");
    if (!std::isfinite(oo->gm_sun) || !std::isfinite(oo->gm_moon) || oo->gm_sun < 0.0 || oo->gm_moon < 0.0)
        return ofail(SRP_EINVAL, "srp_integrate: third-body GM must be finite and >= 0");
    if (oo->gm_sun > 0.0 && !(oo->sun_dist > 0.0)) return ofail(SRP_EINVAL, "srp_integrate: sun_dist must be > 0");
    if (oo->gm_moon > 0.0 && !(oo->moon[0] * oo->moon[0] + oo->moon[1] * oo->moon[1] + oo->moon[2] * oo->moon[2] > 0.0))
        return ofail(SRP_EINVAL, "srp_integrate: the moon position must be non-zero");
    if (n_traj == 0) return SRP_OK;
    if (!z0 || !theta || !zN) return ofail(SRP_EINVAL, "srp_integrate: NULL z0/theta/zN");
    const bool adj = dL_dzN != nullptr;
    if (adj && !dL_dtheta && !dL_dz0) return ofail(SRP_EINVAL, "srp_integrate: adjoint needs dL_dtheta or dL_dz0");
    OCU(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    OrbitDev o;
    std::memset(&o, 0, sizeof o);
    o.mu = oo->mu; o.j2 = oo->j2; o.re = oo->re; o.mass = oo->mass;
    for (int j = 0; j < 3; ++j) { o.I[j] = oo->inertia[j]; o.sun[j] = oo->sun[j]; }
    o.P = oo->pressure; o.dt = oo->dt; o.n_steps = oo->n_steps; o.model = oo->model; o.n_theta = oo->n_theta;
    o.eclipse = oo->eclipse;
    o.gm3[0] = oo->gm_sun; o.gm3[1] = oo->gm_moon;
    for (int j = 0; j < 3; ++j) { o.pos3[0][j] = oo->sun_dist * oo->sun[j]; o.pos3[1][j] = oo->moon[j]; }
    int C = oo->ckpt_every > 0 ? oo->ckpt_every : (int)std::ceil(std::sqrt((double)std::max(1, oo->n_steps)));
    C = std::max(1, std::min(C, kMaxCkptSeg));
    o.ckpt = C;
    std::memcpy(o.in_scale, oo->in_scale, sizeof o.in_scale);
    std::memcpy(o.in_offset, oo->in_offset, sizeof o.in_offset);
    std::memcpy(o.out_mean, oo->out_mean, sizeof o.out_mean);
    std::memcpy(o.out_std, oo->out_std, sizeof o.out_std);
    const int n_ck = oo->n_steps > 0 ? (oo->n_steps + C - 1) / C : 0;
    // device buffers (stream-ordered allocations, freed at the end of the call)
    const int ins[5] = {19, 256, 256, 256, 256}, outs[5] = {256, 256, 256, 256, 6};
    std::vector<void*> allocs;
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), st) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return p;
    };
    auto cleanup = [&]() { for (void* p : allocs) cudaFreeAsync(p, st); allocs.clear(); };
    if (o.model == SRP_FM_PROXY) {
        const float* P = mlp_params_ptr(proxy);
        int64_t off = 0;
        float* wt = (float*)dalloc(sizeof(float) * (size_t)mlp_param_count());
        if (!wt) { cleanup(); return ofail(SRP_ENOMEM, "srp_integrate: scratch"); }
        for (int l = 0; l < 5; ++l) {
            o.W[l] = P + off;
            o.Wt[l] = wt + off;
            transpose_kernel<<<256, 256, 0, st>>>(P + off, wt + off, outs[l], ins[l]);
            off += (int64_t)ins[l] * outs[l];
            o.b[l] = P + off;
            off += outs[l];
        }
    }
#define OCU_FREE(call, where)                                                                          \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            cleanup();                                                                                 \
            return ofail(SRP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_));              \
        }                                                                                              \
    } while (0)
    const double *d_z0 = z0, *d_th = theta, *d_lam = dL_dzN;
    double *d_zN = zN, *d_traj = traj, *d_dth = dL_dtheta, *d_dz0 = dL_dz0;
    const size_t zb = sizeof(double) * 13 * n_traj, tb = sizeof(double) * oo->n_theta * n_traj;
    const size_t trb = sizeof(double) * 13 * (size_t)(oo->n_steps + 1) * n_traj;
    if (mem == SRP_MEM_HOST) {
        double* a = (double*)dalloc(zb); double* b = (double*)dalloc(tb); double* cz = (double*)dalloc(zb);
        if (!a || !b || !cz) { cleanup(); return ofail(SRP_ENOMEM, "srp_integrate: staging"); }
        OCU_FREE(cudaMemcpyAsync(a, z0, zb, cudaMemcpyHostToDevice, st), "H2D z0");
        OCU_FREE(cudaMemcpyAsync(b, theta, tb, cudaMemcpyHostToDevice, st), "H2D theta");
        d_z0 = a; d_th = b; d_zN = cz;
        d_traj = traj ? (double*)dalloc(trb) : nullptr;
        if (adj) {
            double* l = (double*)dalloc(zb);
            if (!l) { cleanup(); return ofail(SRP_ENOMEM, "srp_integrate: staging"); }
            OCU_FREE(cudaMemcpyAsync(l, dL_dzN, zb, cudaMemcpyHostToDevice, st), "H2D lam");
            d_lam = l;
            d_dth = dL_dtheta ? (double*)dalloc(tb) : nullptr;
            d_dz0 = dL_dz0 ? (double*)dalloc(zb) : nullptr;
        }
    } else if (mem != SRP_MEM_DEVICE) {
        cleanup();
        return ofail(SRP_EINVAL, "srp_integrate: bad mem");
    }
    double* ck = adj && n_ck > 0 ? (double*)dalloc(sizeof(double) * 13 * (size_t)n_ck * n_traj) : nullptr;
    // a failed allocation must not reach a kernel as a NULL output
    if ((traj && !d_traj) || (adj && n_ck > 0 && !ck) || (adj && dL_dtheta && !d_dth) ||
        (adj && dL_dz0 && !d_dz0)) {
        cleanup();
        return ofail(SRP_ENOMEM, "srp_integrate: device scratch");
    }
    rk4_forward_kernel<<<n_traj, 256, 0, st>>>(o, d_z0, d_th, d_zN, d_traj, ck, n_ck);
    OCU_FREE(cudaGetLastError(), "rk4 forward launch");
    if (adj) {
        if (n_ck > 0) {
            rk4_adjoint_kernel<<<n_traj, 256, 0, st>>>(o, d_th, ck, n_ck, d_lam, d_dth, d_dz0);
            OCU_FREE(cudaGetLastError(), "rk4 adjoint launch");
        } else {
            if (d_dz0) OCU_FREE(cudaMemcpyAsync(d_dz0, d_lam, zb, cudaMemcpyDeviceToDevice, st), "copy");
            if (d_dth) OCU_FREE(cudaMemsetAsync(d_dth, 0, tb, st), "memset");
        }
    }
    if (mem == SRP_MEM_HOST) {
        OCU_FREE(cudaMemcpyAsync(zN, d_zN, zb, cudaMemcpyDeviceToHost, st), "D2H zN");
        if (traj) OCU_FREE(cudaMemcpyAsync(traj, d_traj, trb, cudaMemcpyDeviceToHost, st), "D2H traj");
        if (adj && dL_dtheta) OCU_FREE(cudaMemcpyAsync(dL_dtheta, d_dth, tb, cudaMemcpyDeviceToHost, st), "D2H dth");
        if (adj && dL_dz0) OCU_FREE(cudaMemcpyAsync(dL_dz0, d_dz0, zb, cudaMemcpyDeviceToHost, st), "D2H dz0");
    }
#undef OCU_FREE
    cleanup();
    if (mem == SRP_MEM_HOST) return srp_sync(c);
    return SRP_OK;
}
