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
// One CTA of 256 threads integrates T trajectories (T = 1, 2, 4 or 8,
// chosen on the host so that the CTAs about fill the GPU).  GB300 issues an
// FP64 warp instruction at a small fraction of the FP32 rate whatever the
// number of active lanes, so the FP64 state algebra of the T trajectories
// runs on T lanes of the same warps (one instruction stream for all of
// them), and every weight the MLP loads serves T queries.  The MLP is
// evaluated by all threads (weights transposed for coalesced reads), in the
// same order of operations for every T, so that a trajectory's result does
// not depend on the batch it was integrated in.  Adjoint: reverse sweep
// over the discrete RK4 map with checkpoints every C steps; a segment is
// recomputed into shared memory and swept backwards.  The vector-Jacobian
// products of the dynamics use forward-mode dual numbers over the same
// templated dyn(): 13 passes seeded on z, 6 on y and 4 on q (for wbar(q)),
// on 23 lanes of warp j for trajectory j; the MLP's input gradient is
// back-propagated by all threads.
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
    double inv_mass, invI[3];             // 1 / mass, 1 / I (host-computed)
    int n_steps, ckpt, model, n_theta;
    int eclipse;                          // cylinder shadow switches SRP off
    double gm3[2], pos3[2][3];            // point masses at fixed positions (GM 0 = off)
    double acc3[2][3];                    // GM s / |s|^3 of each point mass (host-computed)
    float in_scale[19], in_offset[19], out_mean[6], out_std[6];
    // proxy weights (FP32): W_l [out][in], Wt_l [in][out], b_l
    const float* W[5];
    const float* Wt[5];
    const float* b[5];
};

constexpr int kMaxCkptSeg = 64;
constexpr int kOrbitThreads = 256;
// proxy weight loads in flight per thread in the hidden layers (a multiple
// of 4: the partial sums take inputs i = 4m + r in order, whatever the
// chunk, so results do not depend on it)
#ifndef SRP_RK4_WLOADS
#define SRP_RK4_WLOADS 128
#endif
constexpr int kWLoads = SRP_RK4_WLOADS;

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
// 1 / sqrt(a): one square root and one division for value and derivative
// (d/da a^(-1/2) = -a^(-3/2) / 2)
__device__ __forceinline__ double inv_sqrt(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ Dual inv_sqrt(Dual a) {
    const double r = 1.0 / sqrt(a.v);
    return {r, -0.5 * a.d * r * r * r};
}
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

// the dynamics k = f(z, y) for a given force-model output y (6).  The
// gravity terms use 1/|r| (one square root and one division) and its
// powers; the reciprocals of the mass and inertia and the point masses'
// indirect terms come from the host.
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
    const S irn = inv_sqrt(r2);
    const S ir2 = irn * irn;
    const S c1 = cst<S>(-o.mu) * (ir2 * irn);
    const S kj = cst<S>(-1.5 * o.j2 * o.mu * o.re * o.re) * (ir2 * ir2 * irn);
    const S f5 = cst<S>(5.0) * (zz * zz * ir2);
    const S one = cst<S>(1.0), three = cst<S>(3.0);
    const double im = o.inv_mass;
    k[0] = z[3]; k[1] = z[4]; k[2] = z[5];
    k[3] = im * (R00 * F[0] + R01 * F[1] + R02 * F[2]) + c1 * x + kj * x * (one - f5);
    k[4] = im * (R10 * F[0] + R11 * F[1] + R12 * F[2]) + c1 * yy + kj * yy * (one - f5);
    k[5] = im * (R20 * F[0] + R21 * F[1] + R22 * F[2]) + c1 * zz + kj * zz * (three - f5);
    // point masses at fixed positions: GM [(s - r)/|s - r|^3 - s/|s|^3]
    for (int b = 0; b < 2; ++b) {
        if (o.gm3[b] == 0.0) continue;
        const double* sp = o.pos3[b];
        const S dx = cst<S>(sp[0]) - x, dy = cst<S>(sp[1]) - yy, dz = cst<S>(sp[2]) - zz;
        const S id = inv_sqrt(dx * dx + dy * dy + dz * dz);
        const S g = cst<S>(o.gm3[b]) * (id * id * id);
        k[3] = k[3] + g * dx - cst<S>(o.acc3[b][0]);
        k[4] = k[4] + g * dy - cst<S>(o.acc3[b][1]);
        k[5] = k[5] + g * dz - cst<S>(o.acc3[b][2]);
    }
    const S half = cst<S>(0.5);
    k[6] = half * (-(q1 * w0) - q2 * w1 - q3 * w2);
    k[7] = half * (q0 * w0 + q2 * w2 - q3 * w1);
    k[8] = half * (q0 * w1 + q3 * w0 - q1 * w2);
    k[9] = half * (q0 * w2 + q1 * w1 - q2 * w0);
    const S Iw0 = o.I[0] * w0, Iw1 = o.I[1] * w1, Iw2 = o.I[2] * w2;
    k[10] = o.invI[0] * (T[0] - (w1 * Iw2 - w2 * Iw1));
    k[11] = o.invI[1] * (T[1] - (w2 * Iw0 - w0 * Iw2));
    k[12] = o.invI[2] * (T[2] - (w0 * Iw1 - w1 * Iw0));
}

// ---- shared memory of one CTA (T trajectories) ---------------------------------
struct TrajSmem {
    double z[13], u[13], k[4][13];
    double lam[13], zbar[13], kbar[4][13], vj_z[13], vj_th[16], thbar[16];
    double dpass[23];
    double wb[3];
    double theta[16];
    float x[32];  // model input
    float y[8], ybar[8], xbar[32];
};
template <int T>
struct OrbitSmem {
    TrajSmem q[T];
    alignas(16) float zpre[4][256][T];   // hidden pre-activations (trajectory innermost)
    alignas(16) float h[2][256][T];
    alignas(16) float g[2][256][T];      // back-propagated gradients
    double seg[T][kMaxCkptSeg + 1][13];  // adjoint: the recomputed segment
};

// the T values of one feature (contiguous, 4 * T-byte aligned)
template <int T>
__device__ __forceinline__ void ld_t(const float* p, float (&v)[T]) {
    if constexpr (T == 1) {
        v[0] = p[0];
    } else if constexpr (T == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
        for (int q = 0; q < T; q += 4) {
            const float4 a = *reinterpret_cast<const float4*>(p + q);
            v[q] = a.x; v[q + 1] = a.y; v[q + 2] = a.z; v[q + 3] = a.w;
        }
    }
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// y = model(wbar, theta) for the T trajectories; keeps the hidden
// pre-activations for the VJP.  Thread t computes hidden feature t of every
// trajectory: each weight it loads is used T times.  Per trajectory the
// operations and their order do not depend on T (four partial sums over the
// 256 inputs of a hidden layer, a lane-strided sum and a butterfly for the
// outputs).
template <int T>
__device__ void model_fwd(const OrbitDev& o, OrbitSmem<T>& s) {
    const int t = threadIdx.x;
    if (o.model != 2) {  // none / cannonball: lane j of warp 0 for trajectory j
        if (t < T) {
            TrajSmem& q = s.q[t];
            for (int j = 0; j < 6; ++j) q.y[j] = 0.0f;
            if (o.model == 1)
                for (int j = 0; j < 3; ++j) q.y[j] = (float)(-q.theta[0] * q.wb[j]);
        }
        __syncthreads();
        return;
    }
    for (int e = t; e < 19 * T; e += kOrbitThreads) {
        const int j = e / 19, i = e - 19 * j;
        const double xv = i < 3 ? s.q[j].wb[i] : s.q[j].theta[i - 3];
        s.q[j].x[i] = (float)(o.in_scale[i] * xv + o.in_offset[i]);
    }
    __syncthreads();
    {  // layer 0: 19 -> 256
        float a[T];
        const float b0 = o.b[0][t];
#pragma unroll
        for (int j = 0; j < T; ++j) a[j] = b0;
        for (int i = 0; i < 19; ++i) {
            const float w = o.Wt[0][i * 256 + t];
#pragma unroll
            for (int j = 0; j < T; ++j) a[j] = fmaf(w, s.q[j].x[i], a[j]);
        }
#pragma unroll
        for (int j = 0; j < T; ++j) {
            s.zpre[0][t][j] = a[j];
            s.h[0][t][j] = silu_f(a[j]);
        }
    }
    __syncthreads();
    for (int l = 1; l < 4; ++l) {
        const float* hin = &s.h[(l - 1) & 1][0][0];
        const float* Wt = o.Wt[l];
        // kWLoads weight loads in flight per thread and four partial sums:
        // the loop is bound by the latency of the weight stream from L2, so
        // the bytes in flight per SM set its rate (one CTA per SM leaves the
        // registers for them)
        float a[4][T];
        const float bl = o.b[l][t];
#pragma unroll
        for (int j = 0; j < T; ++j) { a[0][j] = bl; a[1][j] = 0.0f; a[2][j] = 0.0f; a[3][j] = 0.0f; }
        for (int i = 0; i < 256; i += kWLoads) {
            float w[kWLoads];
#pragma unroll
            for (int u = 0; u < kWLoads; ++u) w[u] = __ldg(Wt + (i + u) * 256 + t);
#pragma unroll
            for (int u = 0; u < kWLoads; ++u) {
                float hv[T];
                ld_t<T>(hin + (i + u) * T, hv);
#pragma unroll
                for (int j = 0; j < T; ++j) a[u & 3][j] = fmaf(w[u], hv[j], a[u & 3][j]);
            }
        }
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const float z = (a[0][j] + a[1][j]) + (a[2][j] + a[3][j]);
            s.zpre[l][t][j] = z;
            s.h[l & 1][t][j] = silu_f(z);
        }
        __syncthreads();
    }
    {  // layer 4: 256 -> 6, warps 0..5 reduce one output each (all trajectories)
        const int w = t >> 5, lane = t & 31;
        if (w < 6) {
            float a[T];
#pragma unroll
            for (int j = 0; j < T; ++j) a[j] = 0.0f;
            for (int i = lane; i < 256; i += 32) {
                const float wv = o.W[4][w * 256 + i];
                float hv[T];
                ld_t<T>(&s.h[1][i][0], hv);
#pragma unroll
                for (int j = 0; j < T; ++j) a[j] = fmaf(wv, hv[j], a[j]);
            }
#pragma unroll
            for (int j = 0; j < T; ++j) {
                for (int off = 16; off > 0; off >>= 1) a[j] += __shfl_xor_sync(0xffffffffu, a[j], off);
                if (lane == j) s.q[j].y[w] = a[j] + o.b[4][w];
            }
        }
    }
    __syncthreads();
}

// xbar = (d model / d x)^T ybar for the T trajectories: (wbar_bar,
// theta_bar) in q.xbar[0..2], [3..].
template <int T>
__device__ void model_vjp(const OrbitDev& o, OrbitSmem<T>& s) {
    const int t = threadIdx.x;
    if (o.model != 2) {
        if (t < T) {
            TrajSmem& q = s.q[t];
            for (int j = 0; j < 19; ++j) q.xbar[j] = 0.0f;
            if (o.model == 1) {  // y[0:3] = -theta0 wbar
                float tb = 0.0f;
                for (int j = 0; j < 3; ++j) {
                    q.xbar[j] = (float)(-q.theta[0]) * q.ybar[j];
                    tb += (float)(-q.wb[j]) * q.ybar[j];
                }
                q.xbar[3] = tb;
            }
        }
        __syncthreads();
        return;
    }
    {  // dh4[i] = sum_o W4[o][i] ybar[o];  dz3 = dh4 * silu'(z3)
        float a[T];
#pragma unroll
        for (int j = 0; j < T; ++j) a[j] = 0.0f;
        for (int oo = 0; oo < 6; ++oo) {
            const float w = o.W[4][oo * 256 + t];
#pragma unroll
            for (int j = 0; j < T; ++j) a[j] = fmaf(w, s.q[j].ybar[oo], a[j]);
        }
#pragma unroll
        for (int j = 0; j < T; ++j) s.g[0][t][j] = a[j] * dsilu_f(s.zpre[3][t][j]);
    }
    __syncthreads();
    int cur = 0;
    for (int l = 3; l >= 1; --l) {  // dh_l[i] = sum_o W_l[o][i] dz_l[o]; dz_{l-1} = dh_l * silu'(z_{l-1})
        const float* gin = &s.g[cur][0][0];
        const float* W = o.W[l];
        float a[4][T];
#pragma unroll
        for (int j = 0; j < T; ++j) { a[0][j] = 0.0f; a[1][j] = 0.0f; a[2][j] = 0.0f; a[3][j] = 0.0f; }
        for (int oo = 0; oo < 256; oo += kWLoads) {
            float w[kWLoads];
#pragma unroll
            for (int u = 0; u < kWLoads; ++u) w[u] = __ldg(W + (oo + u) * 256 + t);
#pragma unroll
            for (int u = 0; u < kWLoads; ++u) {
                float gv[T];
                ld_t<T>(gin + (oo + u) * T, gv);
#pragma unroll
                for (int j = 0; j < T; ++j) a[u & 3][j] = fmaf(w[u], gv[j], a[u & 3][j]);
            }
        }
#pragma unroll
        for (int j = 0; j < T; ++j)
            s.g[cur ^ 1][t][j] = ((a[0][j] + a[1][j]) + (a[2][j] + a[3][j])) * dsilu_f(s.zpre[l - 1][t][j]);
        __syncthreads();
        cur ^= 1;
    }
    {  // dx[i] = sum_o W0[o][i] dz0[o], i < 19: a warp per (trajectory, input)
        const int w = t >> 5, lane = t & 31;
        for (int e = w; e < 19 * T; e += kOrbitThreads / 32) {
            const int j = e / 19, i = e - 19 * j;
            float a = 0.0f;
            for (int oo = lane; oo < 256; oo += 32) a = fmaf(o.W[0][oo * 19 + i], s.g[cur][oo][j], a);
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) s.q[j].xbar[i] = a * o.in_scale[i];
        }
    }
    __syncthreads();
}

// q.k[stage] = f(q.u) for the T trajectories; leaves wbar and the model
// state in shared memory.  The FP64 algebra runs on lane j of warp 0 for
// trajectory j.
template <int T>
__device__ void feval(const OrbitDev& o, OrbitSmem<T>& s, int stage) {
    const int t = threadIdx.x;
    if (t < T) sun_body<double>(s.q[t].u + 6, o.sun, s.q[t].wb);
    __syncthreads();
    model_fwd<T>(o, s);
    if (t < T) {
        double yd[6];
        for (int j = 0; j < 6; ++j) yd[j] = (double)s.q[t].y[j];
        dyn<double>(o, s.q[t].u, yd, s.q[t].k[stage]);
    }
    __syncthreads();
}

// VJP of f at u = q.u with cotangent q.kbar[stage]: q.vj_z (13) and
// q.vj_th (n_theta), for the T trajectories.  Dual passes of trajectory j
// on lanes 0..22 of warp j.
template <int T>
__device__ void fvjp(const OrbitDev& o, OrbitSmem<T>& s, int stage) {
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    if (t < T) sun_body<double>(s.q[t].u + 6, o.sun, s.q[t].wb);
    __syncthreads();
    model_fwd<T>(o, s);
    // dual passes: 0..12 seed z_i, 13..18 seed y_j, 19..22 seed q_j in wbar(q)
    if (w < T && lane < 19) {
        TrajSmem& q = s.q[w];
        Dual z[13], y[6], k[13];
        for (int j = 0; j < 13; ++j) z[j] = mk(q.u[j], lane == j ? 1.0 : 0.0);
        for (int j = 0; j < 6; ++j) y[j] = mk((double)q.y[j], lane == 13 + j ? 1.0 : 0.0);
        dyn<Dual>(o, z, y, k);
        double acc = 0.0;
        for (int j = 0; j < 13; ++j) acc += q.kbar[stage][j] * k[j].d;
        q.dpass[lane] = acc;
    }
    __syncthreads();
    if (t < 6 * T) {
        const int j = t / 6, c = t - 6 * j;
        s.q[j].ybar[c] = (float)s.q[j].dpass[13 + c];
    }
    __syncthreads();
    model_vjp<T>(o, s);
    // wbar(q) back to q: passes 19..22 seed q_{lane-19}
    if (w < T && lane >= 19 && lane < 23) {
        TrajSmem& q = s.q[w];
        Dual qq[4], wb[3];
        for (int j = 0; j < 4; ++j) qq[j] = mk(q.u[6 + j], (lane - 19) == j ? 1.0 : 0.0);
        sun_body<Dual>(qq, o.sun, wb);
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += (double)q.xbar[j] * wb[j].d;
        q.dpass[lane] = acc;
    }
    __syncthreads();
    if (t < 13 * T) {
        const int j = t / 13, c = t - 13 * j;
        s.q[j].vj_z[c] = s.q[j].dpass[c] + (c >= 6 && c < 10 ? s.q[j].dpass[19 + c - 6] : 0.0);
    }
    if (t < 16 * T) {
        const int j = t / 16, c = t - 16 * j;
        if (c < o.n_theta) s.q[j].vj_th[c] = (double)s.q[j].xbar[3 + c];
    }
    __syncthreads();
}

// one RK4 step q.z -> q.z (in place) for the T trajectories, using q.u, q.k
template <int T>
__device__ void rk4_step(const OrbitDev& o, OrbitSmem<T>& s) {
    const int t = threadIdx.x;
    const double h = o.dt;
    const bool act = t < 13 * T;
    const int j = t / 13, c = t - 13 * j;   // (trajectory, component) when act
    if (act) s.q[j].u[c] = s.q[j].z[c];
    __syncthreads();
    feval<T>(o, s, 0);
    if (act) s.q[j].u[c] = s.q[j].z[c] + 0.5 * h * s.q[j].k[0][c];
    __syncthreads();
    feval<T>(o, s, 1);
    if (act) s.q[j].u[c] = s.q[j].z[c] + 0.5 * h * s.q[j].k[1][c];
    __syncthreads();
    feval<T>(o, s, 2);
    if (act) s.q[j].u[c] = s.q[j].z[c] + h * s.q[j].k[2][c];
    __syncthreads();
    feval<T>(o, s, 3);
    if (act)
        s.q[j].z[c] = s.q[j].z[c] + (h / 6.0) * (s.q[j].k[0][c] + 2.0 * s.q[j].k[1][c] + 2.0 * s.q[j].k[2][c] + s.q[j].k[3][c]);
    __syncthreads();
}

// Trajectories blockIdx.x * T + j, j < T; slots past n_traj integrate a copy
// of the last trajectory and write nothing.
template <int T>
__global__ void __launch_bounds__(kOrbitThreads, 1) rk4_forward_kernel(const OrbitDev o, int n_traj,
                                                                     const double* __restrict__ z0,
                                                                     const double* __restrict__ theta, double* zN,
                                                                     double* traj, double* ckpt, int n_ck) {
    extern __shared__ __align__(16) unsigned char orbit_smem[];
    OrbitSmem<T>& s = *reinterpret_cast<OrbitSmem<T>*>(orbit_smem);
    const int t = threadIdx.x, base = blockIdx.x * T;
    const bool act = t < 13 * T;
    const int j = t / 13, c = t - 13 * j;
    const int tr = min(base + j, n_traj - 1);
    const bool own = act && base + j < n_traj;
    if (act) s.q[j].z[c] = z0[(size_t)tr * 13 + c];
    if (t < 16 * T) {
        const int jj = t / 16, cc = t - 16 * jj;
        if (cc < o.n_theta) s.q[jj].theta[cc] = theta[(size_t)min(base + jj, n_traj - 1) * o.n_theta + cc];
    }
    __syncthreads();
    for (int n = 0; n < o.n_steps; ++n) {
        if (own) {
            if (traj) traj[((size_t)tr * (o.n_steps + 1) + n) * 13 + c] = s.q[j].z[c];
            if (ckpt && n % o.ckpt == 0) ckpt[((size_t)tr * n_ck + n / o.ckpt) * 13 + c] = s.q[j].z[c];
        }
        rk4_step<T>(o, s);
    }
    if (own) {
        if (traj) traj[((size_t)tr * (o.n_steps + 1) + o.n_steps) * 13 + c] = s.q[j].z[c];
        zN[(size_t)tr * 13 + c] = s.q[j].z[c];
    }
}

template <int T>
__global__ void __launch_bounds__(kOrbitThreads, 1) rk4_adjoint_kernel(const OrbitDev o, int n_traj,
                                                                     const double* __restrict__ theta,
                                                                     const double* __restrict__ ckpt, int n_ck,
                                                                     const double* __restrict__ lamN, double* dth,
                                                                     double* dz0) {
    extern __shared__ __align__(16) unsigned char orbit_smem[];
    OrbitSmem<T>& s = *reinterpret_cast<OrbitSmem<T>*>(orbit_smem);
    const int t = threadIdx.x, base = blockIdx.x * T;
    const double h = o.dt;
    const bool act = t < 13 * T;
    const int j = t / 13, c = t - 13 * j;
    const int tr = min(base + j, n_traj - 1);
    const bool own = act && base + j < n_traj;
    const bool tact = t < 16 * T;
    const int tj = t / 16, tc = t - 16 * tj;   // (trajectory, parameter) when tact
    const bool tuse = tact && tc < o.n_theta;
    if (act) s.q[j].lam[c] = lamN[(size_t)tr * 13 + c];
    if (tact) {
        s.q[tj].thbar[tc] = 0.0;
        if (tuse) s.q[tj].theta[tc] = theta[(size_t)min(base + tj, n_traj - 1) * o.n_theta + tc];
    }
    __syncthreads();
    for (int sgi = n_ck - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * o.ckpt;
        const int n1 = min(o.n_steps, n0 + o.ckpt);
        // recompute the segment's states
        if (act) {
            s.seg[j][0][c] = ckpt[((size_t)tr * n_ck + sgi) * 13 + c];
            s.q[j].z[c] = s.seg[j][0][c];
        }
        __syncthreads();
        for (int n = n0; n < n1 - 1; ++n) {
            rk4_step<T>(o, s);
            if (act) s.seg[j][n - n0 + 1][c] = s.q[j].z[c];
            __syncthreads();
        }
        // reverse sweep over the segment
        for (int n = n1 - 1; n >= n0; --n) {
            const int sn = n - n0;
            // stage inputs and slopes
            if (act) s.q[j].u[c] = s.seg[j][sn][c];
            __syncthreads();
            feval<T>(o, s, 0);
            if (act) s.q[j].u[c] = s.seg[j][sn][c] + 0.5 * h * s.q[j].k[0][c];
            __syncthreads();
            feval<T>(o, s, 1);
            if (act) s.q[j].u[c] = s.seg[j][sn][c] + 0.5 * h * s.q[j].k[1][c];
            __syncthreads();
            feval<T>(o, s, 2);
            if (act) {
                TrajSmem& q = s.q[j];
                q.kbar[3][c] = h / 6.0 * q.lam[c];
                q.kbar[2][c] = h / 3.0 * q.lam[c];
                q.kbar[1][c] = h / 3.0 * q.lam[c];
                q.kbar[0][c] = h / 6.0 * q.lam[c];
                q.zbar[c] = q.lam[c];
            }
            __syncthreads();
            // stage 4: u4 = z + h k3
            if (act) s.q[j].u[c] = s.seg[j][sn][c] + h * s.q[j].k[2][c];
            __syncthreads();
            fvjp<T>(o, s, 3);
            if (act) { s.q[j].zbar[c] += s.q[j].vj_z[c]; s.q[j].kbar[2][c] += h * s.q[j].vj_z[c]; }
            if (tuse) s.q[tj].thbar[tc] += s.q[tj].vj_th[tc];
            // stage 3: u3 = z + h/2 k2
            if (act) s.q[j].u[c] = s.seg[j][sn][c] + 0.5 * h * s.q[j].k[1][c];
            __syncthreads();
            fvjp<T>(o, s, 2);
            if (act) { s.q[j].zbar[c] += s.q[j].vj_z[c]; s.q[j].kbar[1][c] += 0.5 * h * s.q[j].vj_z[c]; }
            if (tuse) s.q[tj].thbar[tc] += s.q[tj].vj_th[tc];
            // stage 2: u2 = z + h/2 k1
            if (act) s.q[j].u[c] = s.seg[j][sn][c] + 0.5 * h * s.q[j].k[0][c];
            __syncthreads();
            fvjp<T>(o, s, 1);
            if (act) { s.q[j].zbar[c] += s.q[j].vj_z[c]; s.q[j].kbar[0][c] += 0.5 * h * s.q[j].vj_z[c]; }
            if (tuse) s.q[tj].thbar[tc] += s.q[tj].vj_th[tc];
            // stage 1: u1 = z
            if (act) s.q[j].u[c] = s.seg[j][sn][c];
            __syncthreads();
            fvjp<T>(o, s, 0);
            if (act) { s.q[j].zbar[c] += s.q[j].vj_z[c]; s.q[j].lam[c] = s.q[j].zbar[c]; }
            if (tuse) s.q[tj].thbar[tc] += s.q[tj].vj_th[tc];
            __syncthreads();
        }
    }
    if (own && dz0) dz0[(size_t)tr * 13 + c] = s.q[j].lam[c];
    if (tuse && base + tj < n_traj && dth) dth[(size_t)(base + tj) * o.n_theta + tc] = s.q[tj].thbar[tc];
}

// Wt_l[i][o] = W_l[o][i]
__global__ void transpose_kernel(const float* __restrict__ W, float* __restrict__ Wt, int out, int in) {
    const int64_t n = (int64_t)out * in;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int oo = (int)(e / in), i = (int)(e % in);
        Wt[(int64_t)i * out + oo] = W[e];
    }
}

// Trajectories per CTA: the smallest power of two (at most 8) with which
// the CTAs do not outnumber the SMs.
static int orbit_batch(int n_traj) {
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm < 1)
        return 1;
    const int per = (n_traj + n_sm - 1) / n_sm;
    return per <= 1 ? 1 : per <= 2 ? 2 : per <= 4 ? 4 : 8;
}

// The forward kernel and, when adj and there are checkpoints, the adjoint.
template <int T>
static cudaError_t orbit_launch(const OrbitDev& o, int n_traj, const double* z0, const double* th, double* zN,
                                double* traj, double* ck, int n_ck, bool adj, const double* lam, double* dth,
                                double* dz0, cudaStream_t st) {
    const size_t smem = sizeof(OrbitSmem<T>);
    cudaError_t e = cudaFuncSetAttribute(rk4_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rk4_adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((n_traj + T - 1) / T);
    rk4_forward_kernel<T><<<grid, kOrbitThreads, smem, st>>>(o, n_traj, z0, th, zN, traj, ck, n_ck);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (adj && n_ck > 0) {
        rk4_adjoint_kernel<T><<<grid, kOrbitThreads, smem, st>>>(o, n_traj, th, ck, n_ck, lam, dth, dz0);
        e = cudaGetLastError();
    }
    return e;
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
    o.inv_mass = 1.0 / o.mass;
    for (int j = 0; j < 3; ++j) o.invI[j] = 1.0 / o.I[j];
    for (int b = 0; b < 2; ++b) {
        if (o.gm3[b] == 0.0) continue;
        const double* sp = o.pos3[b];
        const double s2 = sp[0] * sp[0] + sp[1] * sp[1] + sp[2] * sp[2];
        const double gs = o.gm3[b] / (s2 * std::sqrt(s2));
        for (int j = 0; j < 3; ++j) o.acc3[b][j] = gs * sp[j];
    }
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
    const int T = orbit_batch(n_traj);
    OCU_FREE(T == 1   ? orbit_launch<1>(o, n_traj, d_z0, d_th, d_zN, d_traj, ck, n_ck, adj, d_lam, d_dth, d_dz0, st)
             : T == 2 ? orbit_launch<2>(o, n_traj, d_z0, d_th, d_zN, d_traj, ck, n_ck, adj, d_lam, d_dth, d_dz0, st)
             : T == 4 ? orbit_launch<4>(o, n_traj, d_z0, d_th, d_zN, d_traj, ck, n_ck, adj, d_lam, d_dth, d_dz0, st)
                      : orbit_launch<8>(o, n_traj, d_z0, d_th, d_zN, d_traj, ck, n_ck, adj, d_lam, d_dth, d_dz0, st),
             "rk4 launch");
    if (adj) {
        if (n_ck == 0) {
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
