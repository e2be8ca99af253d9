/*
 * srp_oracle.c -- FP64 CPU oracle of the solar-radiation-pressure (SRP)
 * ray-grid estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The product library
 * (the CUDA path) shares no code, header, table or constant with it.
 *
 * What it computes (paper, Sec. 3.2):
 *   force  F(w,theta) = integral over the surface M(theta) of the force
 *                       field f(x,w,theta)                     (Eq. Force/F)
 *   torque tau(w,theta) = integral over M of (x - x_COM) x f   (Eq. torque)
 * with the light-to-force map l2f (Sec. 3.2): photons arriving along the
 * travel direction d transfer their momentum; reflected photons carry
 * momentum away along w_out.  The estimator is a grid of parallel rays
 * over the bounding sphere (the "ray-grid" family of Sec. 2.1 / Table
 * "Methods"), with closest hits found by testing every ray against EVERY
 * triangle (the paper's own brute-force intersection, Sec. 3.2,
 * "Estimation").  No acceleration structure is used.
 *
 * Steps, in order, per ray i of sun direction s of design index D:
 *  1. Philox4x32-10 (Salmon et al., SC'11) with counter (i, s, D, k) and key
 *     (seed_lo, seed_hi); uniform u(x) = (x >> 8) * 2^-24.
 *  2. Orthonormal basis (u,v) of the travel direction d = -e by the
 *     branchless construction of Duff et al. 2017.
 *  3. Grid over the square of side 2R centred on the mesh's AABB centre c,
 *     R = max |vertex - c|: pixel (px,py) with jitter (xi1,xi2) (or 0.5),
 *     origin o = c + (-R+(px+xi1)dx) u + (-R+(py+xi2)dy) v - 2R d,
 *     per-ray momentum weight w0 = P dx dy.
 *  4. Closest hit over all triangles, watertight ray/triangle test of Woop,
 *     Benthin and Wald (JCGT 2013), FP64.  Ties on t go to the smaller
 *     triangle index.  Bounce rays skip their source triangle and hits with
 *     t <= 1e-6 R.
 *  5. At hit k (normal flipped to face the ray, cos = -n.d):
 *       k == K:  deposit w [(1-rs) d - (2 rs cos + 2/3 rd) n]   (expected
 *                value of the reflection, the per-plate law)
 *       k <  K:  branch with fixed probability 1/2 (xi_b = u(x0)):
 *                specular r = d - 2(d.n)n,        w' = 2 w rs
 *                diffuse  cosine-weighted about n, w' = 2 w rd
 *                         (direction of n + s, s uniform on the unit
 *                         sphere from (u(x1), u(x2)))
 *                deposit w d - w' d'; continue with (x, d', w')
 *     torque deposit (x - COM) x deposit.  Rays that miss deposit nothing.
 *  6. Sums in FP64 in ray order k.  Uncertainty: each pixel is one
 *     stratum with one sample, so the variance of the total is estimated by
 *     collapsing neighbouring strata in pairs (k = 2j, 2j+1) (Cochran,
 *     "Sampling Techniques", collapsed strata): var = sum_j (y_2j - y_2j+1)^2,
 *     plus y^2 of an unpaired last ray; sigma = sqrt(var) per component.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* 1. Philox4x32-10, from its published definition (Salmon et al. 2011) */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void rng4(uint64_t seed, uint32_t i, uint32_t s, uint32_t dsg, uint32_t k, double u[4])
{
    uint32_t ctr[4] = {i, s, dsg, k};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    for (int j = 0; j < 4; ++j) u[j] = u24(o[j]);
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3])
{
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}

/* 2. Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin (2017):
 *    branchless ONB for a unit vector n; (b1, b2, n) right-handed. */
void or_onb(const double n[3], double b1[3], double b2[3])
{
    double sign = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* ------------------------------------------------------------------ */
/* 4. Watertight ray/triangle intersection (Woop, Benthin, Wald 2013)  */
/* ------------------------------------------------------------------ */
typedef struct {
    double o[3], d[3];
    int kx, ky, kz;
    double Sx, Sy, Sz;
} wray;

static void wray_setup(wray* r, const double o[3], const double d[3])
{
    for (int j = 0; j < 3; ++j) { r->o[j] = o[j]; r->d[j] = d[j]; }
    int kz = 0;
    double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    if (ay > ax && ay >= az) kz = 1;
    else if (az > ax && az > ay) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) { int t = kx; kx = ky; ky = t; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = d[kx] / d[kz]; r->Sy = d[ky] / d[kz]; r->Sz = 1.0 / d[kz];
}

/* Returns 1 and the ray parameter t when the ray hits the triangle. */
static int wray_hit(const wray* r, const double* p0, const double* p1, const double* p2, double* t_out)
{
    double A[3], B[3], C[3];
    for (int j = 0; j < 3; ++j) { A[j] = p0[j] - r->o[j]; B[j] = p1[j] - r->o[j]; C[j] = p2[j] - r->o[j]; }
    const int kx = r->kx, ky = r->ky, kz = r->kz;
    double Ax = A[kx] - r->Sx * A[kz], Ay = A[ky] - r->Sy * A[kz];
    double Bx = B[kx] - r->Sx * B[kz], By = B[ky] - r->Sy * B[kz];
    double Cx = C[kx] - r->Sx * C[kz], Cy = C[ky] - r->Sy * C[kz];
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double Az = r->Sz * A[kz], Bz = r->Sz * B[kz], Cz = r->Sz * C[kz];
    double T = U * Az + V * Bz + W * Cz;
    *t_out = T / det;
    return 1;
}

/* ------------------------------------------------------------------ */
/* scene                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int T;
    const double* tv;      /* [T][9] vertex positions (double)          */
    const double* tn;      /* [T][3] unit geometric normal (e1 x e2)    */
    const int32_t* group;  /* [T]                                        */
    const double* rho;     /* [G][2]                                     */
    double c[3], R;        /* grid centre (AABB centre) and radius       */
    double com[3];
    double P;
    int nx, ny, K, jitter;
    uint64_t seed;
    uint32_t dsg;          /* design index used in the RNG counter       */
} scene_t;

/* Closest hit by brute force: smallest t > tmin, ties -> smaller index. */
static int closest(const scene_t* sc, const wray* r, double tmin, int skip, double* t_best)
{
    int best = -1;
    double tb = INFINITY;
    for (int f = 0; f < sc->T; ++f) {
        if (f == skip) continue;
        const double* v = sc->tv + 9 * (size_t)f;
        double t;
        if (!wray_hit(r, v, v + 3, v + 6, &t)) continue;
        if (!(t > tmin)) continue;
        if (t < tb) { tb = t; best = f; }
    }
    *t_best = tb;
    return best;
}

/* Per-path record, used by the gradient. */
typedef struct {
    int m;              /* number of hits (segments that hit)            */
    int f[8];           /* hit triangle                                   */
    int br[8];          /* 0 specular, 1 diffuse (k < K only)            */
    double w[9];        /* weight arriving at hit k                      */
    double x[8][3];     /* hit point                                     */
    double d[8][3];     /* arriving direction                            */
    double n[8][3];     /* facing normal                                 */
    double cs[8];       /* cos = -n.d                                    */
    double dout[8][3];  /* outgoing direction (k < K)                    */
    double us[8][3];    /* diffuse branch: the uniform unit-sphere point */
} path_t;

static void grid_ray(const scene_t* sc, const double e[3], uint64_t i, uint32_t s,
                     double o[3], double d[3], double* w0)
{
    for (int j = 0; j < 3; ++j) d[j] = -e[j];
    double bu[3], bv[3];
    or_onb(d, bu, bv);
    uint32_t px = (uint32_t)(i % (uint64_t)sc->nx), py = (uint32_t)(i / (uint64_t)sc->nx);
    double xi1 = 0.5, xi2 = 0.5;
    if (sc->jitter) {
        double u[4];
        rng4(sc->seed, (uint32_t)i, s, sc->dsg, 0, u);
        xi1 = u[0]; xi2 = u[1];
    }
    double dx = 2.0 * sc->R / sc->nx, dy = 2.0 * sc->R / sc->ny;
    double a = -sc->R + ((double)px + xi1) * dx;
    double b = -sc->R + ((double)py + xi2) * dy;
    for (int j = 0; j < 3; ++j) o[j] = sc->c[j] + a * bu[j] + b * bv[j] - 2.0 * sc->R * d[j];
    *w0 = sc->P * dx * dy;
}

/* Trace one ray path; accumulate force/torque (6) into acc; fill path. */
static void trace_path(const scene_t* sc, const double e[3], uint64_t i, uint32_t s,
                       double acc[6], path_t* pth)
{
    double o[3], d[3], w;
    grid_ray(sc, e, i, s, o, d, &w);
    int src = -1;
    double tmin = 0.0;
    pth->m = 0;
    for (int k = 1; k <= sc->K; ++k) {
        wray r;
        wray_setup(&r, o, d);
        double t;
        int f = closest(sc, &r, tmin, src, &t);
        if (f < 0) break;
        int h = k - 1;
        pth->m = k;
        pth->f[h] = f;
        pth->w[h] = w;
        double x[3], n[3];
        for (int j = 0; j < 3; ++j) x[j] = o[j] + t * d[j];
        const double* ng = sc->tn + 3 * (size_t)f;
        double sgn = dot3(ng, d) > 0.0 ? -1.0 : 1.0;
        for (int j = 0; j < 3; ++j) n[j] = sgn * ng[j];
        double cs = -dot3(n, d);
        const double rs = sc->rho[2 * sc->group[f]], rd = sc->rho[2 * sc->group[f] + 1];
        for (int j = 0; j < 3; ++j) { pth->x[h][j] = x[j]; pth->d[h][j] = d[j]; pth->n[h][j] = n[j]; }
        pth->cs[h] = cs;
        double dp[3], arm[3], tq[3];
        for (int j = 0; j < 3; ++j) arm[j] = x[j] - sc->com[j];
        if (k == sc->K) {
            double cn = 2.0 * rs * cs + (2.0 / 3.0) * rd;
            for (int j = 0; j < 3; ++j) dp[j] = w * ((1.0 - rs) * d[j] - cn * n[j]);
            cross3(arm, dp, tq);
            for (int j = 0; j < 3; ++j) { acc[j] += dp[j]; acc[3 + j] += tq[j]; }
            break;
        }
        double u[4];
        rng4(sc->seed, (uint32_t)i, s, sc->dsg, (uint32_t)k, u);
        double dout[3], wout;
        if (u[0] < 0.5) {
            for (int j = 0; j < 3; ++j) dout[j] = d[j] + 2.0 * cs * n[j];
            wout = 2.0 * w * rs;
            pth->br[h] = 0;
        } else {
            /* Lambertian reflection: the direction from x to a uniform point
             * on the unit sphere centred at x + n is cosine-distributed about
             * n (pdf cos/pi); no tangent frame is needed. */
            double z = 1.0 - 2.0 * u[1], rr = sqrt(fmax(0.0, 1.0 - z * z)), phi = 2.0 * M_PI * u[2];
            double v[3] = {n[0] + rr * cos(phi), n[1] + rr * sin(phi), n[2] + z};
            double L = sqrt(dot3(v, v));
            for (int j = 0; j < 3; ++j) dout[j] = L > 0.0 ? v[j] / L : n[j];
            wout = 2.0 * w * rd;
            pth->br[h] = 1;
            pth->us[h][0] = rr * cos(phi); pth->us[h][1] = rr * sin(phi); pth->us[h][2] = z;
        }
        for (int j = 0; j < 3; ++j) { dp[j] = w * d[j] - wout * dout[j]; pth->dout[h][j] = dout[j]; }
        cross3(arm, dp, tq);
        for (int j = 0; j < 3; ++j) { acc[j] += dp[j]; acc[3 + j] += tq[j]; }
        pth->w[h + 1] = wout;
        for (int j = 0; j < 3; ++j) { o[j] = x[j]; d[j] = dout[j]; }
        w = wout;
        src = f;
        tmin = 1e-6 * sc->R;
    }
}

/* ------------------------------------------------------------------ */
/* Reverse-mode gradient of one path's contribution L = sum_k q_k.dp_k */
/* (rho part: exact along the fixed path; hinge part: K == 1, hit      */
/* point held fixed on its facet, see or_force_grad).                  */
/* ------------------------------------------------------------------ */
static void path_grad(const scene_t* sc, const path_t* p, const double gF[3], const double gT[3],
                      double* d_rho /*[G][2]*/)
{
    if (p->m == 0) return;
    double wbar_next = 0.0;  /* adjoint of w_{h+1} */
    for (int h = p->m - 1; h >= 0; --h) {
        const int f = p->f[h];
        const int g = sc->group[f];
        const double rs = sc->rho[2 * g], rd = sc->rho[2 * g + 1];
        double arm[3], q[3];
        for (int j = 0; j < 3; ++j) arm[j] = p->x[h][j] - sc->com[j];
        cross3(gT, arm, q);
        for (int j = 0; j < 3; ++j) q[j] += gF[j];
        const double w = p->w[h];
        double wbar;
        if (h + 1 == sc->K) {
            /* closed-form deposit w[(1-rs)d - (2 rs c + 2/3 rd) n] */
            double qd = dot3(q, p->d[h]), qn = dot3(q, p->n[h]);
            double cs = p->cs[h];
            d_rho[2 * g] += w * (-qd - 2.0 * cs * qn);
            d_rho[2 * g + 1] += w * (-(2.0 / 3.0) * qn);
            wbar = (1.0 - rs) * qd - (2.0 * rs * cs + (2.0 / 3.0) * rd) * qn;
        } else {
            /* deposit w d - w' d'; w' = 2 w rho_branch */
            double wbar_out = wbar_next - dot3(q, p->dout[h]);
            wbar = dot3(q, p->d[h]);
            double rb = p->br[h] == 0 ? rs : rd;
            d_rho[2 * g + p->br[h]] += wbar_out * 2.0 * w;
            wbar += wbar_out * 2.0 * rb;
        }
        wbar_next = wbar;
    }
}

/* Rotation of v about the unit axis a by angle ang (Rodrigues). */
static void rotate(const double a[3], double ang, const double v[3], double o[3])
{
    double c = cos(ang), s = sin(ang), axv[3];
    cross3(a, v, axv);
    double ad = dot3(a, v);
    for (int j = 0; j < 3; ++j) o[j] = v[j] * c + axv[j] * s + a[j] * ad * (1.0 - c);
}

/* Value of a recorded path's contribution L = sum_k q_k . dp_k with hinge
 * hh turned by `ang`, in the fixed-visibility reading of the hinge
 * derivative: the path keeps its facets, its branch choices and its random
 * draws, and the facets on hinge hh turn with it.  The primary hit point is
 * carried by its facet (as at K = 1: weight w c(ang) / c0); every later hit
 * is the intersection of the outgoing ray with the plane of the same facet
 * (its recorded facing normal, turned if the facet turns); the outgoing
 * direction follows the turned normal (specular: d + 2 c n; diffuse: the
 * same uniform sphere point u, direction (n + u) / |n + u|).  At ang = 0 it
 * reproduces the path's own deposits. */
static double path_value_hinge(const scene_t* sc, const path_t* p, const double gF[3], const double gT[3],
                               const int32_t* thinge, int hh, const double ap[3], const double aa[3], double ang)
{
    double x[3], n[3], d[3], rel[3], o[3];
    const int f0 = p->f[0];
    for (int j = 0; j < 3; ++j) { x[j] = p->x[0][j]; n[j] = p->n[0][j]; d[j] = p->d[0][j]; }
    if (thinge[f0] == hh) {
        for (int j = 0; j < 3; ++j) rel[j] = x[j] - ap[j];
        rotate(aa, ang, rel, o);
        for (int j = 0; j < 3; ++j) x[j] = o[j] + ap[j];
        rotate(aa, ang, p->n[0], n);
    }
    double c = -dot3(n, d);
    double w = p->w[0] * c / p->cs[0];
    double L = 0.0;
    for (int k = 0; k < p->m; ++k) {
        const int g = sc->group[p->f[k]];
        const double rs = sc->rho[2 * g], rd = sc->rho[2 * g + 1];
        double arm[3], q[3], dp[3];
        for (int j = 0; j < 3; ++j) arm[j] = x[j] - sc->com[j];
        cross3(gT, arm, q);
        for (int j = 0; j < 3; ++j) q[j] += gF[j];
        if (k + 1 == sc->K) {
            const double cn = 2.0 * rs * c + (2.0 / 3.0) * rd;
            for (int j = 0; j < 3; ++j) dp[j] = w * ((1.0 - rs) * d[j] - cn * n[j]);
            L += dot3(q, dp);
            break;
        }
        double dout[3], wout;
        if (p->br[k] == 0) {
            for (int j = 0; j < 3; ++j) dout[j] = d[j] + 2.0 * c * n[j];
            wout = 2.0 * w * rs;
        } else {
            double v[3];
            for (int j = 0; j < 3; ++j) v[j] = n[j] + p->us[k][j];
            const double Ln = sqrt(dot3(v, v));
            for (int j = 0; j < 3; ++j) dout[j] = Ln > 0.0 ? v[j] / Ln : n[j];
            wout = 2.0 * w * rd;
        }
        for (int j = 0; j < 3; ++j) dp[j] = w * d[j] - wout * dout[j];
        L += dot3(q, dp);
        if (k + 1 >= p->m) break;   /* the outgoing ray left the craft */
        const int f1 = p->f[k + 1];
        double v0[3], n1[3];
        for (int j = 0; j < 3; ++j) { v0[j] = sc->tv[9 * (size_t)f1 + j]; n1[j] = p->n[k + 1][j]; }
        if (thinge[f1] == hh) {
            for (int j = 0; j < 3; ++j) rel[j] = v0[j] - ap[j];
            rotate(aa, ang, rel, o);
            for (int j = 0; j < 3; ++j) v0[j] = o[j] + ap[j];
            double nt[3];
            rotate(aa, ang, n1, nt);
            for (int j = 0; j < 3; ++j) n1[j] = nt[j];
        }
        for (int j = 0; j < 3; ++j) rel[j] = v0[j] - x[j];
        const double t = dot3(n1, rel) / dot3(n1, dout);
        for (int j = 0; j < 3; ++j) { x[j] += t * dout[j]; n[j] = n1[j]; d[j] = dout[j]; }
        c = -dot3(n, d);
        w = wout;
    }
    return L;
}

/* Step of the central difference of path_value_hinge (radians). */
#define OR_HINGE_STEP 1e-6

/* Hinge derivative of a K=1 hit: the ray's surface element is carried
 * rigidly by the facet, so the ray's contribution is (w/c0) c(a) q.G(n(a)). */
static double hinge_term(const scene_t* sc, const path_t* p, const double gF[3], const double gT[3],
                         const double axis_p[3], const double axis_a[3])
{
    const int f = p->f[0];
    const int g = sc->group[f];
    const double rs = sc->rho[2 * g], rd = sc->rho[2 * g + 1];
    const double* x = p->x[0];
    const double* n = p->n[0];
    const double* d = p->d[0];
    const double c = p->cs[0];
    double arm[3], q[3], Gv[3], dn[3], dx[3], rel[3], dq[3], dG[3];
    for (int j = 0; j < 3; ++j) { arm[j] = x[j] - sc->com[j]; rel[j] = x[j] - axis_p[j]; }
    cross3(gT, arm, q);
    for (int j = 0; j < 3; ++j) q[j] += gF[j];
    const double cn = 2.0 * rs * c + (2.0 / 3.0) * rd;
    for (int j = 0; j < 3; ++j) Gv[j] = (1.0 - rs) * d[j] - cn * n[j];
    cross3(axis_a, n, dn);        /* dn/da */
    cross3(axis_a, rel, dx);      /* dx/da */
    const double dc = -dot3(dn, d);
    cross3(gT, dx, dq);           /* dq/da */
    for (int j = 0; j < 3; ++j) dG[j] = -2.0 * rs * dc * n[j] - cn * dn[j];
    const double dphi = dc * dot3(q, Gv) + c * (dot3(dq, Gv) + dot3(q, dG));
    return (p->w[0] / c) * dphi;
}

/* ------------------------------------------------------------------ */
/* threaded driver                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    const scene_t* sc;
    const double* sun;     /* [S][3] */
    int S;
    int64_t off, stride, n;
    int64_t chunk;         /* rays per job (even) */
    int64_t nchunk;
    uint32_t sun_base;
    double* part;          /* [S][nchunk][12]: sums (6), squared pair diffs (6) */
    /* gradient */
    const double* up;      /* [S][6] or NULL */
    const double* hp;      /* [H][6] hinge axes */
    const int32_t* thinge; /* [T] */
    int H, G;
    double* grad_rho;      /* per-thread [G][2] */
    double* grad_h;        /* per-thread [H] */
    int64_t job0, job1;    /* jobs = s*nchunk + c */
} work_t;

static void* worker(void* arg)
{
    work_t* wk = (work_t*)arg;
    const scene_t* sc = wk->sc;
    path_t p;
    for (int64_t job = wk->job0; job < wk->job1; ++job) {
        int s = (int)(job / wk->nchunk);
        int64_t c = job % wk->nchunk;
        const double* e = wk->sun + 3 * (size_t)s;
        double acc[6] = {0, 0, 0, 0, 0, 0}, sq[6] = {0, 0, 0, 0, 0, 0}, pend[6] = {0, 0, 0, 0, 0, 0};
        int64_t k0 = c * wk->chunk, k1 = k0 + wk->chunk < wk->n ? k0 + wk->chunk : wk->n;
        for (int64_t k = k0; k < k1; ++k) {
            uint64_t i = (uint64_t)(wk->off + k * wk->stride);
            double y[6] = {0, 0, 0, 0, 0, 0};
            trace_path(sc, e, i, wk->sun_base + (uint32_t)s, y, &p);
            for (int j = 0; j < 6; ++j) acc[j] += y[j];
            if ((k & 1) == 0) {
                for (int j = 0; j < 6; ++j) pend[j] = y[j];
                if (k + 1 == wk->n) for (int j = 0; j < 6; ++j) sq[j] += y[j] * y[j];
            } else {
                for (int j = 0; j < 6; ++j) { double q = y[j] - pend[j]; sq[j] += q * q; }
            }
            if (wk->up) {
                const double* g6 = wk->up + 6 * (size_t)s;
                path_grad(sc, &p, g6, g6 + 3, wk->grad_rho);
                if (wk->H > 0 && sc->K == 1 && p.m == 1) {
                    int hh = wk->thinge[p.f[0]];
                    if (hh >= 0)
                        wk->grad_h[hh] += hinge_term(sc, &p, g6, g6 + 3, wk->hp + 6 * hh, wk->hp + 6 * hh + 3);
                } else if (wk->H > 0 && sc->K > 1) {
                    /* every hinge that turns a facet of the path: central
                     * difference of the fixed-visibility path value */
                    for (int k = 0; k < p.m; ++k) {
                        const int hh = wk->thinge[p.f[k]];
                        if (hh < 0 || hh >= wk->H) continue;
                        int dup = 0;
                        for (int k2 = 0; k2 < k; ++k2) dup |= wk->thinge[p.f[k2]] == hh;
                        if (dup) continue;
                        const double* ap = wk->hp + 6 * hh;
                        const double vp = path_value_hinge(sc, &p, g6, g6 + 3, wk->thinge, hh, ap, ap + 3, OR_HINGE_STEP);
                        const double vm = path_value_hinge(sc, &p, g6, g6 + 3, wk->thinge, hh, ap, ap + 3, -OR_HINGE_STEP);
                        wk->grad_h[hh] += (vp - vm) / (2.0 * OR_HINGE_STEP);
                    }
                }
            }
        }
        double* dst = wk->part + 12 * ((size_t)s * wk->nchunk + c);
        for (int j = 0; j < 6; ++j) { dst[j] = acc[j]; dst[6 + j] = sq[j]; }
    }
    return NULL;
}

static void build_scene(scene_t* sc, double* tv, double* tn, const float* verts, int V,
                        const int32_t* tris, int T)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < V; ++v)
        for (int j = 0; j < 3; ++j) {
            double x = verts[3 * v + j];
            if (x < lo[j]) lo[j] = x;
            if (x > hi[j]) hi[j] = x;
        }
    for (int j = 0; j < 3; ++j) sc->c[j] = 0.5 * (lo[j] + hi[j]);
    double R2 = 0.0;
    for (int v = 0; v < V; ++v) {
        double r2 = 0.0;
        for (int j = 0; j < 3; ++j) { double q = verts[3 * v + j] - sc->c[j]; r2 += q * q; }
        if (r2 > R2) R2 = r2;
    }
    sc->R = sqrt(R2);
    for (int f = 0; f < T; ++f) {
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j) tv[9 * f + 3 * c + j] = verts[3 * tris[3 * f + c] + j];
        double e1[3], e2[3], nn[3];
        for (int j = 0; j < 3; ++j) { e1[j] = tv[9 * f + 3 + j] - tv[9 * f + j]; e2[j] = tv[9 * f + 6 + j] - tv[9 * f + j]; }
        cross3(e1, e2, nn);
        double l = sqrt(dot3(nn, nn));
        for (int j = 0; j < 3; ++j) tn[3 * f + j] = l > 0.0 ? nn[j] / l : 0.0;
    }
    sc->T = T;
    sc->tv = tv;
    sc->tn = tn;
}

/* Grid parameters (centre c, radius R) as the oracle defines them. */
void or_grid(const float* verts, int V, double c_out[3], double* R_out)
{
    int32_t tri0[3] = {0, 0, 0};
    double tv[9], tn[3];
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tri0, V > 0 ? 1 : 0);
    for (int j = 0; j < 3; ++j) c_out[j] = sc.c[j];
    *R_out = sc.R;
}

/*
 * Force/torque of one design for S sun directions.
 *   verts [V][3] f32, tris [T][3], group [T], rho [G][2] (f64),
 *   sun [S][3] unit vectors toward the sun, com [3].
 *   Ray subset: k = 0..n-1 traces grid ray i = off + k*stride
 *   (n = 0: the full grid, off = 0, stride = 1).
 *   out_ft [S][6] (F, tau), out_sigma [S][6] or NULL.
 *   Gradient (optional, up != NULL): upstream dL/d(F,tau) [S][6];
 *   d_rho [G][2] and d_hinge [H] are ADDED to.  Hinges: K = 1 the
 *   analytic derivative of hinge_term; K > 1 the central difference of
 *   path_value_hinge (fixed visibility) per path.
 */
int or_force(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
             const double* rho, int G, const double* sun, int S, const double* com,
             int nx, int ny, int K, int jitter, uint64_t seed, double P,
             int64_t off, int64_t stride, int64_t n, uint32_t sun_base, uint32_t dsg,
             int threads, double* out_ft, double* out_sigma,
             const double* up, const int32_t* thinge, const double* hinge_axes, int H,
             double* d_rho, double* d_hinge)
{
    if (T < 0 || V < 0 || S < 0 || nx <= 0 || ny <= 0 || K < 1 || K > 8) return 1;
    if (n <= 0) { off = 0; stride = 1; n = (int64_t)nx * ny; }
    if (threads <= 0) threads = 1;
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.group = group; sc.rho = rho;
    for (int j = 0; j < 3; ++j) sc.com[j] = com[j];
    sc.P = P; sc.nx = nx; sc.ny = ny; sc.K = K; sc.jitter = jitter; sc.seed = seed; sc.dsg = dsg;
    const int64_t chunk = 4096;
    const int64_t nchunk = (n + chunk - 1) / chunk;
    double* part = (double*)calloc((size_t)S * nchunk * 12 + 1, sizeof(double));
    int64_t jobs = (int64_t)S * nchunk;
    if (threads > jobs) threads = jobs > 0 ? (int)jobs : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    work_t* wk = (work_t*)calloc(threads, sizeof(work_t));
    double* gr = up ? (double*)calloc((size_t)threads * (2 * G + H + 1), sizeof(double)) : NULL;
    for (int t = 0; t < threads; ++t) {
        wk[t].sc = &sc; wk[t].sun = sun; wk[t].S = S;
        wk[t].off = off; wk[t].stride = stride; wk[t].n = n;
        wk[t].chunk = chunk; wk[t].nchunk = nchunk;
        wk[t].sun_base = sun_base; wk[t].part = part;
        wk[t].up = up; wk[t].hp = hinge_axes; wk[t].thinge = thinge; wk[t].H = H; wk[t].G = G;
        if (gr) { wk[t].grad_rho = gr + (size_t)t * (2 * G + H + 1); wk[t].grad_h = wk[t].grad_rho + 2 * G; }
        wk[t].job0 = jobs * t / threads;
        wk[t].job1 = jobs * (t + 1) / threads;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, worker, &wk[t]);
    worker(&wk[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    for (int s = 0; s < S; ++s) {
        double tot[12] = {0};
        for (int64_t c = 0; c < nchunk; ++c)
            for (int j = 0; j < 12; ++j) tot[j] += part[12 * ((size_t)s * nchunk + c) + j];
        if (out_ft) for (int j = 0; j < 6; ++j) out_ft[6 * s + j] = tot[j];
        if (out_sigma) for (int j = 0; j < 6; ++j) out_sigma[6 * s + j] = sqrt(tot[6 + j]);
    }
    if (gr) {
        for (int t = 0; t < threads; ++t) {
            for (int q = 0; q < 2 * G; ++q) d_rho[q] += wk[t].grad_rho[q];
            for (int h = 0; h < H; ++h) d_hinge[h] += wk[t].grad_h[h];
        }
    }
    free(gr); free(wk); free(th); free(part); free(tv); free(tn);
    return 0;
}

/*
 * Finite-difference companion of the hinge gradient: the SAME estimator
 * with each K=1 hit carried rigidly by its facet, re-evaluated at hinge
 * angle offsets +-h by rotating (x, n) about the hinge axis, without
 * re-tracing.  Returns the central difference of L = sum_s up_s.(F_s,tau_s)
 * in d_hinge[H].  Single-threaded; for small test cases.
 */

int or_hinge_fd_fixed_hits(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                           const double* rho, int G, const double* sun, int S, const double* com,
                           int nx, int ny, int jitter, uint64_t seed, double P,
                           const double* up, const int32_t* thinge, const double* hinge_axes, int H,
                           double hstep, double* d_hinge)
{
    (void)G;
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.group = group; sc.rho = rho;
    for (int j = 0; j < 3; ++j) sc.com[j] = com[j];
    sc.P = P; sc.nx = nx; sc.ny = ny; sc.K = 1; sc.jitter = jitter; sc.seed = seed; sc.dsg = 0;
    for (int h = 0; h < H; ++h) d_hinge[h] = 0.0;
    path_t p;
    int64_t n = (int64_t)nx * ny;
    for (int s = 0; s < S; ++s) {
        const double* e = sun + 3 * s;
        const double* gF = up + 6 * s;
        const double* gT = up + 6 * s + 3;
        for (int64_t i = 0; i < n; ++i) {
            double acc[6] = {0};
            trace_path(&sc, e, (uint64_t)i, (uint32_t)s, acc, &p);
            if (p.m != 1) continue;
            int hh = thinge[p.f[0]];
            if (hh < 0) continue;
            const double* ap = hinge_axes + 6 * hh;
            const double* aa = ap + 3;
            const int g = group[p.f[0]];
            const double rs = rho[2 * g], rd = rho[2 * g + 1];
            double val[2];
            for (int sg = 0; sg < 2; ++sg) {
                double ang = sg == 0 ? hstep : -hstep;
                double rel[3], xr[3], nr[3], arm[3], q[3], dp[3];
                for (int j = 0; j < 3; ++j) rel[j] = p.x[0][j] - ap[j];
                rotate(aa, ang, rel, xr);
                rotate(aa, ang, p.n[0], nr);
                for (int j = 0; j < 3; ++j) { xr[j] += ap[j]; arm[j] = xr[j] - com[j]; }
                double c = -dot3(nr, p.d[0]);
                double wa = p.w[0] / p.cs[0] * c;
                double cn = 2.0 * rs * c + (2.0 / 3.0) * rd;
                for (int j = 0; j < 3; ++j) dp[j] = wa * ((1.0 - rs) * p.d[0][j] - cn * nr[j]);
                cross3(gT, arm, q);
                for (int j = 0; j < 3; ++j) q[j] += gF[j];
                val[sg] = dot3(q, dp);
            }
            d_hinge[hh] += (val[0] - val[1]) / (2.0 * hstep);
        }
    }
    free(tv); free(tn);
    return 0;
}

/* Single-ray debug query: hit triangle of the primary ray (or -1) and t. */
int or_primary_hit(const float* verts, int V, const int32_t* tris, int T, const double* sun,
                   int nx, int ny, int jitter, uint64_t seed, uint32_t sun_idx, uint32_t dsg,
                   int64_t i, double* t_out)
{
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.nx = nx; sc.ny = ny; sc.jitter = jitter; sc.seed = seed; sc.dsg = dsg; sc.P = 1.0;
    double o[3], d[3], w;
    grid_ray(&sc, sun, (uint64_t)i, sun_idx, o, d, &w);
    wray r;
    wray_setup(&r, o, d);
    int f = closest(&sc, &r, 0.0, -1, t_out);
    free(tv); free(tn);
    return f;
}

/* Per-ray samples: for each listed grid ray index, the ray's force and
 * torque deposits out_y [n][6] and the original index of the triangle hit
 * at each bounce out_hits [n][K] (-1 after the path ends). */
typedef struct {
    const scene_t* sc;
    const double* sun;
    uint32_t sun_idx;
    const int64_t* idx;
    int64_t q0, q1;
    double* out_y;
    int32_t* out_hits;
} rays_job;

static void* rays_worker(void* arg)
{
    rays_job* j = (rays_job*)arg;
    path_t p;
    const int K = j->sc->K;
    for (int64_t q = j->q0; q < j->q1; ++q) {
        double y[6] = {0, 0, 0, 0, 0, 0};
        trace_path(j->sc, j->sun, (uint64_t)j->idx[q], j->sun_idx, y, &p);
        for (int c = 0; c < 6; ++c) j->out_y[6 * q + c] = y[c];
        for (int k = 0; k < K; ++k) j->out_hits[q * K + k] = k < p.m ? p.f[k] : -1;
    }
    return NULL;
}

int or_trace_rays(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                  const double* rho, const double* sun, const double* com,
                  int nx, int ny, int K, int jitter, uint64_t seed, double P,
                  uint32_t sun_idx, uint32_t dsg, const int64_t* idx, int64_t n,
                  double* out_y, int32_t* out_hits, int threads)
{
    if (K < 1 || K > 8) return 1;
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.group = group; sc.rho = rho;
    for (int j = 0; j < 3; ++j) sc.com[j] = com[j];
    sc.P = P; sc.nx = nx; sc.ny = ny; sc.K = K; sc.jitter = jitter; sc.seed = seed; sc.dsg = dsg;
    if (threads < 1) threads = 1;
    if (threads > n) threads = n > 0 ? (int)n : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    rays_job* jb = (rays_job*)calloc(threads, sizeof(rays_job));
    for (int t = 0; t < threads; ++t) {
        jb[t].sc = &sc; jb[t].sun = sun; jb[t].sun_idx = sun_idx; jb[t].idx = idx;
        jb[t].q0 = n * t / threads; jb[t].q1 = n * (t + 1) / threads;
        jb[t].out_y = out_y; jb[t].out_hits = out_hits;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, rays_worker, &jb[t]);
    rays_worker(&jb[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    free(jb); free(th); free(tv); free(tn);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Area-sampling estimator with next-event estimation (the paper's own  */
/* estimator, Sec. 3.2 "Estimation", without bounces):                 */
/*  - triangle f (original order) receives n_f = max(1, ceil(rho A_f))  */
/*    samples, A_f and the product computed in FP32 with every         */
/*    operation rounded (the integer count is a floating-point          */
/*    decision: both sides take it in FP32);                           */
/*  - sample j: Philox counter (j, f, sun, design | 2^31), uniform point */
/*    on the triangle x = v0 + s(1-u2) e1 + s u2 e2, s = sqrt(u1)       */
/*    (Osada, Funkhouser, Chazelle, Dobkin 2002);                       */
/*  - facing normal n (n.e >= 0), cos = n.e; shadow ray from x toward   */
/*    the sun (skip f, t > 1e-6 R): visible -> deposit                  */
/*    (A_f / n_f) P cos [(1-rs) d - (2 rs cos + 2/3 rd) n], d = -e,      */
/*    torque (x - COM) x deposit;                                       */
/*  - sums in sample order k = prefix(f) + j; sigma: collapsed strata   */
/*    over pairs (k = 2i, 2i+1).                                        */
/*  With K = 2 each sample also gathers one Lambertian interreflection  */
/*  (the indirect term of the estimator: a BRDF-sampled incoming         */
/*  direction, its closest hit y, next-event estimation at y):          */
/*  - per side sigma = +1, -1 of the facet (n_s = sigma n_e, n_e the     */
/*    winding normal): direction omega = unit(n_s + s), s uniform on the */
/*    unit sphere (cosine-distributed about n_s, pdf cos/pi); side +1    */
/*    takes (u2, u3) of the sample's counter, side -1 (u0, u1) of the    */
/*    counter (j, f, sun, design | 2^31 | 2^28);                         */
/*  - closest hit y of the ray (x, omega) (skip f, t > 1e-6 R); y's side */
/*    that faces x, m, is lit when m.e > 0 and the shadow ray from y     */
/*    along e (skip y's triangle, t > 1e-6 R) is free;                   */
/*  - the radiance y reflects toward x is rd_y P (m.e) / pi, so the      */
/*    irradiance estimate at x is E = pi L / pdf * cos = rd_y P (m.e);   */
/*  - x receives that light arriving along -omega at cos = omega.n_s and */
/*    deposits (A_f / n_f) E [(1-rs) (-omega) - (2 rs cos + 2/3 rd) n_s] */
/*    (its own BRDF, the per-plate law), torque about COM.               */
/*  Only y's diffuse reflection is gathered: its specular reflection is  */
/*  a delta lobe that a sampled direction reaches with probability 0.    */
/* ------------------------------------------------------------------ */
static float area32(const double* tv)
{
    float a0 = (float)tv[0], a1 = (float)tv[1], a2 = (float)tv[2];
    float e1x = (float)tv[3] - a0, e1y = (float)tv[4] - a1, e1z = (float)tv[5] - a2;
    float e2x = (float)tv[6] - a0, e2y = (float)tv[7] - a1, e2z = (float)tv[8] - a2;
    float p, q;
    p = e1y * e2z; q = e1z * e2y; float cx = p - q;
    p = e1z * e2x; q = e1x * e2z; float cy = p - q;
    p = e1x * e2y; q = e1y * e2x; float cz = p - q;
    float s = cx * cx; s = s + cy * cy; s = s + cz * cz;
    return 0.5f * sqrtf(s);
}

int64_t or_area_counts(const float* verts, int V, const int32_t* tris, int T, float density, int32_t* counts)
{
    double tv[9];
    int64_t tot = 0;
    for (int f = 0; f < T; ++f) {
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j) tv[3 * c + j] = verts[3 * tris[3 * f + c] + j];
        float a = area32(tv);
        float prod = density * a;
        int32_t n = (int32_t)ceilf(prod);
        if (n < 1) n = 1;
        counts[f] = n;
        tot += n;
    }
    (void)V;
    return tot;
}

typedef struct {
    const scene_t* sc;
    const double* sun;
    const int32_t* counts;
    const int64_t* prefix;
    int S;
    uint32_t sun_base;
    int K;              /* 1: direct light only; 2: plus one Lambertian interreflection */
    double* out;        /* [S][12] */
    int s0, s1;
} area_job;

/* One gathered Lambertian interreflection at x (side normal ns, winding
 * facet f) along omega = unit(ns + uniform unit vector(ua, ub)); adds the
 * deposit and torque to y6.  wA = A_f / n_f, (rs, rd) of the facet of x. */
static void gather_diffuse(const scene_t* sc, const double e[3], int f, const double x[3], const double ns[3],
                           double ua, double ub, double wA, double rs, double rd, double y6[6])
{
    double z = 1.0 - 2.0 * ua, rr = sqrt(fmax(0.0, 1.0 - z * z)), phi = 2.0 * M_PI * ub;
    double om[3] = {ns[0] + rr * cos(phi), ns[1] + rr * sin(phi), ns[2] + z};
    double L = sqrt(dot3(om, om));
    if (!(L > 0.0)) return;
    for (int q = 0; q < 3; ++q) om[q] /= L;
    wray r;
    wray_setup(&r, x, om);
    double t;
    const int h = closest(sc, &r, 1e-6 * sc->R, f, &t);
    if (h < 0) return;
    const double* nh = sc->tn + 3 * (size_t)h;
    double m[3];
    double sg = dot3(nh, om) > 0.0 ? -1.0 : 1.0;          /* the side of y facing x */
    for (int q = 0; q < 3; ++q) m[q] = sg * nh[q];
    const double ce = dot3(m, e);
    if (!(ce > 0.0)) return;
    double yp[3];
    for (int q = 0; q < 3; ++q) yp[q] = x[q] + t * om[q];
    wray rs_;
    wray_setup(&rs_, yp, e);
    double ts;
    if (closest(sc, &rs_, 1e-6 * sc->R, h, &ts) >= 0) return;
    const double E = sc->rho[2 * sc->group[h] + 1] * sc->P * ce;
    const double cs = dot3(om, ns);
    const double cn = 2.0 * rs * cs + (2.0 / 3.0) * rd;
    double dp[3], arm[3], tq[3];
    for (int q = 0; q < 3; ++q) { dp[q] = wA * E * (-(1.0 - rs) * om[q] - cn * ns[q]); arm[q] = x[q] - sc->com[q]; }
    cross3(arm, dp, tq);
    for (int q = 0; q < 3; ++q) { y6[q] += dp[q]; y6[3 + q] += tq[q]; }
}

static void* area_worker(void* arg)
{
    area_job* jb = (area_job*)arg;
    const scene_t* sc = jb->sc;
    for (int s = jb->s0; s < jb->s1; ++s) {
        const double* e = jb->sun + 3 * (size_t)s;
        double d[3] = {-e[0], -e[1], -e[2]};
        double acc[6] = {0}, sq[6] = {0}, pend[6] = {0};
        int64_t k = 0;
        for (int f = 0; f < sc->T; ++f) {
            const double* v = sc->tv + 9 * (size_t)f;
            double e1[3], e2[3];
            for (int j = 0; j < 3; ++j) { e1[j] = v[3 + j] - v[j]; e2[j] = v[6 + j] - v[j]; }
            double cr[3];
            cross3(e1, e2, cr);
            const double A = 0.5 * sqrt(dot3(cr, cr));
            const double* ng = sc->tn + 3 * (size_t)f;
            double n[3];
            double sg = dot3(ng, e) < 0.0 ? -1.0 : 1.0;
            for (int j = 0; j < 3; ++j) n[j] = sg * ng[j];
            const double cs = dot3(n, e);
            const double rs = sc->rho[2 * sc->group[f]], rd = sc->rho[2 * sc->group[f] + 1];
            const int32_t nf = jb->counts[f];
            const double wgt = sc->P * A / nf;
            for (int32_t j = 0; j < nf; ++j, ++k) {
                double u[4];
                uint32_t ctr[4] = {(uint32_t)j, (uint32_t)f, jb->sun_base + (uint32_t)s, sc->dsg | 0x80000000u};
                uint32_t key[2] = {(uint32_t)sc->seed, (uint32_t)(sc->seed >> 32)};
                uint32_t o[4];
                or_philox4x32_10(ctr, key, o);
                for (int q = 0; q < 4; ++q) u[q] = u24(o[q]);
                const double ss = sqrt(u[0]);
                const double b1 = ss * (1.0 - u[1]), b2 = ss * u[1];
                double x[3];
                for (int q = 0; q < 3; ++q) x[q] = v[q] + b1 * e1[q] + b2 * e2[q];
                double y[6] = {0, 0, 0, 0, 0, 0};
                if (cs > 0.0) {
                    wray r;
                    wray_setup(&r, x, e);
                    double t;
                    const int hit = closest(sc, &r, 1e-6 * sc->R, f, &t);
                    if (hit < 0) {
                        const double cn = 2.0 * rs * cs + (2.0 / 3.0) * rd;
                        double dp[3], arm[3], tq[3];
                        for (int q = 0; q < 3; ++q) { dp[q] = wgt * cs * ((1.0 - rs) * d[q] - cn * n[q]); arm[q] = x[q] - sc->com[q]; }
                        cross3(arm, dp, tq);
                        for (int q = 0; q < 3; ++q) { y[q] = dp[q]; y[3 + q] = tq[q]; }
                    }
                }
                if (jb->K >= 2) {
                    /* both sides of the facet gather one interreflection */
                    const double wA = A / nf;
                    double ns[3];
                    for (int q = 0; q < 3; ++q) ns[q] = ng[q];
                    gather_diffuse(sc, e, f, x, ns, u[2], u[3], wA, rs, rd, y);
                    uint32_t ctr2[4] = {(uint32_t)j, (uint32_t)f, jb->sun_base + (uint32_t)s,
                                        sc->dsg | 0x80000000u | 0x10000000u};
                    uint32_t key2[2] = {(uint32_t)sc->seed, (uint32_t)(sc->seed >> 32)};
                    uint32_t o2[4];
                    or_philox4x32_10(ctr2, key2, o2);
                    for (int q = 0; q < 3; ++q) ns[q] = -ng[q];
                    gather_diffuse(sc, e, f, x, ns, u24(o2[0]), u24(o2[1]), wA, rs, rd, y);
                }
                for (int q = 0; q < 6; ++q) acc[q] += y[q];
                if ((k & 1) == 0) {
                    for (int q = 0; q < 6; ++q) pend[q] = y[q];
                } else {
                    for (int q = 0; q < 6; ++q) { double dd = y[q] - pend[q]; sq[q] += dd * dd; }
                }
            }
        }
        if (k & 1) for (int q = 0; q < 6; ++q) sq[q] += pend[q] * pend[q];
        for (int q = 0; q < 6; ++q) { jb->out[12 * s + q] = acc[q]; jb->out[12 * s + 6 + q] = sq[q]; }
    }
    return NULL;
}

int or_force_area(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                  const double* rho, const double* sun, int S, const double* com, float density,
                  uint64_t seed, double P, uint32_t sun_base, uint32_t dsg, int K, int threads,
                  double* out_ft, double* out_sigma)
{
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    int32_t* counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.group = group; sc.rho = rho;
    for (int j = 0; j < 3; ++j) sc.com[j] = com[j];
    sc.P = P; sc.seed = seed; sc.dsg = dsg; sc.K = 1;
    or_area_counts(verts, V, tris, T, density, counts);
    double* out = (double*)calloc((size_t)S * 12 + 1, sizeof(double));
    if (threads < 1) threads = 1;
    if (threads > S) threads = S > 0 ? S : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    area_job* jb = (area_job*)calloc(threads, sizeof(area_job));
    for (int t = 0; t < threads; ++t) {
        jb[t].sc = &sc; jb[t].sun = sun; jb[t].counts = counts; jb[t].S = S; jb[t].sun_base = sun_base; jb[t].K = K;
        jb[t].out = out; jb[t].s0 = S * t / threads; jb[t].s1 = S * (t + 1) / threads;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, area_worker, &jb[t]);
    area_worker(&jb[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    for (int s = 0; s < S; ++s)
        for (int q = 0; q < 6; ++q) {
            out_ft[6 * s + q] = out[12 * s + q];
            if (out_sigma) out_sigma[6 * s + q] = sqrt(out[12 * s + 6 + q]);
        }
    free(jb); free(th); free(out); free(counts); free(tv); free(tn);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Local Lambertian thermal emitters (Sec. 5.9 "Design": heat from      */
/* on-board compute radiated as a Lambertian source, recoil factor 2/3  */
/* of a collimated beam):                                               */
/*  - triangles of group g emit on the side of their winding normal     */
/*    n_e = unit(e1 x e2) with momentum flux P * emit[g] per unit area  */
/*    (emit in W/m^2 and P = 1/c gives newtons);                        */
/*  - triangle f with emit > 0 receives n_f = max(1, ceil(rho A_f))     */
/*    samples (FP32 as for the area estimator), others none;            */
/*  - sample j: Philox counter (j, f, 0, design | 2^30); point from      */
/*    (u0, u1) as in or_force_area; direction omega = unit(n_e + s),     */
/*    s the uniform unit vector of (u2, u3) (cosine-distributed about    */
/*    n_e); packet momentum w = P emit A_f / n_f;                       */
/*  - recoil: the packet's expected recoil -(2/3) w n_e at x (the mean   */
/*    of -w omega), torque (x - com) x recoil;                          */
/*  - the packet's ray (skip f, t > 1e-6 R) deposits at its closest hit  */
/*    y the closed form w[(1-rs) omega - (2 rs cos + 2/3 rd) n], n the   */
/*    hit normal facing the ray, cos = -n.omega; torque (y - com) x it;  */
/*  - sums in sample order k = prefix(f) + j; sigma: collapsed strata.   */
/* ------------------------------------------------------------------ */
int64_t or_thermal_counts(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                          const float* emit, float density, int32_t* counts)
{
    double tv[9];
    int64_t tot = 0;
    for (int f = 0; f < T; ++f) {
        if (!(emit[group[f]] > 0.0f)) { counts[f] = 0; continue; }
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j) tv[3 * c + j] = verts[3 * tris[3 * f + c] + j];
        float a = area32(tv);
        float prod = density * a;
        int32_t n = (int32_t)ceilf(prod);
        if (n < 1) n = 1;
        counts[f] = n;
        tot += n;
    }
    (void)V;
    return tot;
}

typedef struct {
    const scene_t* sc;
    const float* emit;
    const int32_t* counts;
    const int64_t* prefix;
    double* y;          /* [N][6] */
    int f0, f1;
} thermal_job;

static void* thermal_worker(void* arg)
{
    thermal_job* jb = (thermal_job*)arg;
    const scene_t* sc = jb->sc;
    for (int f = jb->f0; f < jb->f1; ++f) {
        const int32_t nf = jb->counts[f];
        if (nf == 0) continue;
        const double* v = sc->tv + 9 * (size_t)f;
        double e1[3], e2[3], cr[3];
        for (int j = 0; j < 3; ++j) { e1[j] = v[3 + j] - v[j]; e2[j] = v[6 + j] - v[j]; }
        cross3(e1, e2, cr);
        const double A = 0.5 * sqrt(dot3(cr, cr));
        const double* ne = sc->tn + 3 * (size_t)f;
        const double w = sc->P * (double)jb->emit[sc->group[f]] * A / nf;
        for (int32_t j = 0; j < nf; ++j) {
            double* y = jb->y + 6 * (size_t)(jb->prefix[f] + j);
            double u[4];
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)f, 0u, sc->dsg | 0x40000000u};
            uint32_t key[2] = {(uint32_t)sc->seed, (uint32_t)(sc->seed >> 32)};
            uint32_t o[4];
            or_philox4x32_10(ctr, key, o);
            for (int q = 0; q < 4; ++q) u[q] = u24(o[q]);
            const double ss = sqrt(u[0]);
            const double b1 = ss * (1.0 - u[1]), b2 = ss * u[1];
            double x[3], arm[3], rc[3], tq[3];
            for (int q = 0; q < 3; ++q) x[q] = v[q] + b1 * e1[q] + b2 * e2[q];
            for (int q = 0; q < 3; ++q) { rc[q] = -(2.0 / 3.0) * w * ne[q]; arm[q] = x[q] - sc->com[q]; }
            cross3(arm, rc, tq);
            for (int q = 0; q < 3; ++q) { y[q] = rc[q]; y[3 + q] = tq[q]; }
            /* cosine-distributed direction: unit(n_e + uniform unit vector) */
            double z = 1.0 - 2.0 * u[2], rr = sqrt(fmax(0.0, 1.0 - z * z)), phi = 2.0 * M_PI * u[3];
            double om[3] = {ne[0] + rr * cos(phi), ne[1] + rr * sin(phi), ne[2] + z};
            double L = sqrt(dot3(om, om));
            if (!(L > 0.0)) continue;
            for (int q = 0; q < 3; ++q) om[q] /= L;
            wray r;
            wray_setup(&r, x, om);
            double t;
            const int h = closest(sc, &r, 1e-6 * sc->R, f, &t);
            if (h < 0) continue;
            const double* nh = sc->tn + 3 * (size_t)h;
            double n[3];
            double sg = dot3(nh, om) > 0.0 ? -1.0 : 1.0;
            for (int q = 0; q < 3; ++q) n[q] = sg * nh[q];
            const double cs = -dot3(n, om);
            const double rs = sc->rho[2 * sc->group[h]], rd = sc->rho[2 * sc->group[h] + 1];
            const double cn = 2.0 * rs * cs + (2.0 / 3.0) * rd;
            double yh[3], dp[3];
            for (int q = 0; q < 3; ++q) {
                yh[q] = x[q] + t * om[q];
                dp[q] = w * ((1.0 - rs) * om[q] - cn * n[q]);
                arm[q] = yh[q] - sc->com[q];
            }
            cross3(arm, dp, tq);
            for (int q = 0; q < 3; ++q) { y[q] += dp[q]; y[3 + q] += tq[q]; }
        }
    }
    return NULL;
}

int or_force_thermal(const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                     const double* rho, const float* emit, const double* com, float density, uint64_t seed,
                     double P, uint32_t dsg, int threads, double* out_ft, double* out_sigma, int64_t* out_n)
{
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    int32_t* counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
    int64_t* prefix = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    scene_t sc;
    memset(&sc, 0, sizeof sc);
    build_scene(&sc, tv, tn, verts, V, tris, T);
    sc.group = group; sc.rho = rho;
    for (int j = 0; j < 3; ++j) sc.com[j] = com[j];
    sc.P = P; sc.seed = seed; sc.dsg = dsg; sc.K = 1;
    const int64_t N = or_thermal_counts(verts, V, tris, group, T, emit, density, counts);
    int64_t acc_n = 0;
    for (int f = 0; f < T; ++f) { prefix[f] = acc_n; acc_n += counts[f]; }
    double* y = (double*)calloc((size_t)(N > 0 ? N : 1) * 6, sizeof(double));
    if (threads < 1) threads = 1;
    if (threads > T) threads = T > 0 ? T : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    thermal_job* jb = (thermal_job*)calloc(threads, sizeof(thermal_job));
    for (int t = 0; t < threads; ++t) {
        jb[t].sc = &sc; jb[t].emit = emit; jb[t].counts = counts; jb[t].prefix = prefix; jb[t].y = y;
        jb[t].f0 = (int)((int64_t)T * t / threads); jb[t].f1 = (int)((int64_t)T * (t + 1) / threads);
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, thermal_worker, &jb[t]);
    thermal_worker(&jb[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    double acc[6] = {0}, sq[6] = {0};
    for (int64_t k = 0; k < N; ++k) {
        const double* yk = y + 6 * (size_t)k;
        for (int q = 0; q < 6; ++q) acc[q] += yk[q];
        if (k & 1) {
            for (int q = 0; q < 6; ++q) { double dd = yk[q] - yk[q - 6]; sq[q] += dd * dd; }
        }
    }
    if (N & 1) for (int q = 0; q < 6; ++q) sq[q] += y[6 * (size_t)(N - 1) + q] * y[6 * (size_t)(N - 1) + q];
    for (int q = 0; q < 6; ++q) { out_ft[q] = acc[q]; if (out_sigma) out_sigma[q] = sqrt(sq[q]); }
    if (out_n) *out_n = N;
    free(jb); free(th); free(y); free(prefix); free(counts); free(tv); free(tn);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Per-sample designs (the paper's training-data sampler, Sec. 3.2      */
/* "Estimation" and Alg. 1 NNLoss: every sample has its own design and  */
/* sun direction; intersection by brute force over its triangles):       */
/*  - sample s instantiates the base mesh with its hinge angles          */
/*    angles[s][H] (Rodrigues in FP64, rounded to float32);              */
/*  - its ray is the single jittered pixel of a 1 x 1 grid over the      */
/*    square of side 2R about the given centre c (c, R must bound every  */
/*    design): Philox counter (0, sample_base + s, 2^29, k), weight       */
/*    P (2R)^2; then the grid estimator's path (K bounces) with the      */
/*    sample's reflectances rho[s][G][2] and torque reference com[s];    */
/*  - out_y[s][6] is the sample's (F, tau) estimate, out_hits[s][K] the   */
/*    hit triangles (-1 after the path ends).                             */
/* ------------------------------------------------------------------ */
static void rot_hinge(const double* hinge, double angle, double R[9])
{
    const double* a = hinge + 3;
    const double nrm = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double x = a[0] / nrm, y = a[1] / nrm, z = a[2] / nrm;
    const double c = cos(angle), s = sin(angle), t = 1.0 - c;
    R[0] = c + x * x * t;     R[1] = x * y * t - z * s; R[2] = x * z * t + y * s;
    R[3] = y * x * t + z * s; R[4] = c + y * y * t;     R[5] = y * z * t - x * s;
    R[6] = z * x * t - y * s; R[7] = z * y * t + x * s; R[8] = c + z * z * t;
}

typedef struct {
    const float* verts; int V; const int32_t* vhinge; const double* hinges; int H;
    const int32_t* tris; const int32_t* group; int T;
    const double* angles; const double* rho; int G; const double* sun; const double* com;
    const double* center; double R; int K; uint64_t seed; double P; uint32_t sample_base;
    double* out_y; int32_t* out_hits;
    int64_t s0, s1;
} samp_job;

static void* samp_worker(void* arg)
{
    samp_job* jb = (samp_job*)arg;
    float* v = (float*)malloc(sizeof(float) * 3 * (size_t)(jb->V > 0 ? jb->V : 1));
    double* tv = (double*)malloc(sizeof(double) * 9 * (size_t)(jb->T > 0 ? jb->T : 1));
    double* tn = (double*)malloc(sizeof(double) * 3 * (size_t)(jb->T > 0 ? jb->T : 1));
    double* Rm = (double*)malloc(sizeof(double) * 9 * (size_t)(jb->H > 0 ? jb->H : 1));
    for (int64_t s = jb->s0; s < jb->s1; ++s) {
        for (int h = 0; h < jb->H; ++h) rot_hinge(jb->hinges + 6 * h, jb->angles[(size_t)s * jb->H + h], Rm + 9 * h);
        for (int q = 0; q < jb->V; ++q) {
            const int h = jb->H > 0 ? jb->vhinge[q] : -1;
            if (h < 0) { for (int j = 0; j < 3; ++j) v[3 * q + j] = jb->verts[3 * q + j]; continue; }
            const double* p = jb->hinges + 6 * h;
            const double* R = Rm + 9 * h;
            const double w[3] = {jb->verts[3 * q] - p[0], jb->verts[3 * q + 1] - p[1], jb->verts[3 * q + 2] - p[2]};
            for (int j = 0; j < 3; ++j) v[3 * q + j] = (float)(p[j] + R[3 * j] * w[0] + R[3 * j + 1] * w[1] + R[3 * j + 2] * w[2]);
        }
        scene_t sc;
        memset(&sc, 0, sizeof sc);
        build_scene(&sc, tv, tn, v, jb->V, jb->tris, jb->T);
        for (int j = 0; j < 3; ++j) { sc.c[j] = jb->center[j]; sc.com[j] = jb->com[3 * (size_t)s + j]; }
        sc.R = jb->R;
        sc.group = jb->group;
        sc.rho = jb->rho + (size_t)s * jb->G * 2;
        sc.P = jb->P; sc.nx = 1; sc.ny = 1; sc.K = jb->K; sc.jitter = 1;
        sc.seed = jb->seed; sc.dsg = 0x20000000u;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        path_t pth;
        trace_path(&sc, jb->sun + 3 * (size_t)s, 0u, jb->sample_base + (uint32_t)s, acc, &pth);
        for (int q = 0; q < 6; ++q) jb->out_y[6 * (size_t)s + q] = acc[q];
        if (jb->out_hits)
            for (int k = 0; k < jb->K; ++k) jb->out_hits[(size_t)s * jb->K + k] = k < pth.m ? pth.f[k] : -1;
    }
    free(v); free(tv); free(tn); free(Rm);
    return NULL;
}

int or_trace_samples(const float* verts, int V, const int32_t* vhinge, const double* hinges, int H,
                     const int32_t* tris, const int32_t* group, int T, const double* angles, const double* rho, int G,
                     const double* sun, const double* com, int64_t N, const double* center, double R, int K,
                     uint64_t seed, double P, uint32_t sample_base, int threads, double* out_y, int32_t* out_hits)
{
    if (threads < 1) threads = 1;
    if (threads > N) threads = N > 0 ? (int)N : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    samp_job* jb = (samp_job*)calloc(threads, sizeof(samp_job));
    for (int t = 0; t < threads; ++t) {
        samp_job j = {verts, V, vhinge, hinges, H, tris, group, T, angles, rho, G, sun, com, center, R, K, seed, P,
                      sample_base, out_y, out_hits, N * t / threads, N * (t + 1) / threads};
        jb[t] = j;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, samp_worker, &jb[t]);
    samp_worker(&jb[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    free(jb); free(th);
    return 0;
}
