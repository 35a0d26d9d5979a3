/*
 * oracle.c -- FP64 reference of the per-frame particle update (arXiv 2504.18056).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU baseline. It shares no code with the CUDA path.
 *
 * Every function is written for a reader checking it against the paper by eye:
 * loops in the order the definitions give, no blocking, no fusion. Build with
 * -ffp-contract=off so that float decisions (neighbour selection) use separate
 * IEEE multiplies and adds.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* SE(3)                                                                     */
/* ------------------------------------------------------------------------ */

void ora_pose_mul(const double A[12], const double B[12], double C[12]) {
    double out[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double s = (c == 3) ? A[r * 4 + 3] : 0.0;
            for (int k = 0; k < 3; ++k) s += A[r * 4 + k] * B[k * 4 + c];
            out[r * 4 + c] = s;
        }
    }
    memcpy(C, out, sizeof(out));
}

void ora_pose_inv(const double A[12], double B[12]) {
    double out[12];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) out[r * 4 + c] = A[c * 4 + r];
    for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s -= out[r * 4 + k] * A[k * 4 + 3];
        out[r * 4 + 3] = s;
    }
    memcpy(B, out, sizeof(out));
}

static void hat(const double w[3], double W[9]) {
    W[0] = 0;     W[1] = -w[2]; W[2] = w[1];
    W[3] = w[2];  W[4] = 0;     W[5] = -w[0];
    W[6] = -w[1]; W[7] = w[0];  W[8] = 0;
}

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    double o[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[r * 3 + k] * B[k * 3 + c];
            o[r * 3 + c] = s;
        }
    memcpy(C, o, sizeof(o));
}

/* exp of xi = [omega; v]: R = I + a W + b W^2, V = I + b W + c W^2, t = V v with
 * a = sin(th)/th, b = (1-cos th)/th^2, c = (th - sin th)/th^3 (Rodrigues and the
 * left Jacobian of SO(3)); their Taylor series below th = 1e-4, and for c below
 * th = 0.1, where the closed form cancels. */
void ora_se3_exp(const double xi[6], double T[12]) {
    const double *w = xi, *v = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b, c;
    if (th < 1e-4) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        double sh = sin(0.5 * th) / th;
        a = sin(th) / th;
        b = 2.0 * sh * sh;                    /* (1 - cos th)/th^2 without cancellation */
        if (th < 0.1)                         /* (th - sin th)/th^3 by its series */
            c = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0 - th2 * th2 * th2 / 362880.0;
        else
            c = (th - sin(th)) / (th2 * th);
    }
    double W[9], W2[9];
    hat(w, W);
    mat3_mul(W, W, W2);
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + a * W[i] + b * W2[i];
        V[i] = I + b * W[i] + c * W2[i];
    }
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) T[r * 4 + k] = R[r * 3 + k];
        T[r * 4 + 3] = V[r * 3 + 0] * v[0] + V[r * 3 + 1] * v[1] + V[r * 3 + 2] * v[2];
    }
}

/* log: th = acos((tr R - 1)/2), omega = th/(2 sin th) vee(R - R^T), v = V^-1 t,
 * V^-1 = I - W/2 + (1 - a/(2b))/th^2 W^2. Valid away from th = pi. */
void ora_se3_log(const double T[12], double xi[6]) {
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[r * 3 + c] = T[r * 4 + c];
    double ct = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double th = acos(ct);
    double k = (th < 1e-6) ? 0.5 + th * th / 12.0 : th / (2.0 * sin(th));
    double w[3] = {k * (R[7] - R[5]), k * (R[2] - R[6]), k * (R[3] - R[1])};
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double thn = sqrt(th2);
    double coef;
    if (thn < 0.1) {
        coef = 1.0 / 12.0 + th2 / 720.0 + th2 * th2 / 30240.0;
    } else {
        double a = sin(thn) / thn, b = (1.0 - cos(thn)) / th2;
        coef = (1.0 - a / (2.0 * b)) / th2;
    }
    double W[9], W2[9];
    hat(w, W);
    mat3_mul(W, W, W2);
    double t[3] = {T[3], T[7], T[11]};
    for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int c = 0; c < 3; ++c) {
            double I = (r == c) ? 1.0 : 0.0;
            s += (I - 0.5 * W[r * 3 + c] + coef * W2[r * 3 + c]) * t[c];
        }
        xi[3 + r] = s;
    }
    xi[0] = w[0]; xi[1] = w[1]; xi[2] = w[2];
}

/* Right Jacobian of SE(3): exp(xi + d) = exp(xi) exp(Jr(xi) d + O(d^2)). With
 * xi = [omega; v] it is Jl(-xi), and the left Jacobian in this order is
 * [[J, 0], [Q, J]] with J the SO(3) left Jacobian I + b W + c W^2 and, for
 * rho = v, phi = omega (Barfoot, State Estimation for Robotics, Sec. 7.1.5),
 *   Q = rho^/2 + c1 (phi^ rho^ + rho^ phi^ + phi^ rho^ phi^)
 *       + c2 (phi^ phi^ rho^ + rho^ phi^ phi^ - 3 phi^ rho^ phi^)
 *       + c3 (phi^ rho^ phi^ phi^ + phi^ phi^ rho^ phi^),
 *   c1 = (th - sin th)/th^3, c2 = (th^2 + 2 cos th - 2)/(2 th^4),
 *   c3 = (2 th - 3 sin th + th cos th)/(2 th^5); power series below th = 0.1. */
void ora_se3_jr(const double xi[6], double J[36]) {
    double phi[3] = {-xi[0], -xi[1], -xi[2]}, rho[3] = {-xi[3], -xi[4], -xi[5]};
    double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double th = sqrt(th2);
    double b, c1, c2, c3;
    if (th < 0.1) {
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        c1 = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0 - th2 * th2 * th2 / 362880.0;
        c2 = 1.0 / 24.0 - th2 / 720.0 + th2 * th2 / 40320.0;
        c3 = 1.0 / 120.0 - th2 / 2520.0 + th2 * th2 / 120960.0;
    } else {
        double s = sin(th), c = cos(th);
        b = (1.0 - c) / th2;
        c1 = (th - s) / (th2 * th);
        c2 = (th2 + 2.0 * c - 2.0) / (2.0 * th2 * th2);
        c3 = (2.0 * th - 3.0 * s + th * c) / (2.0 * th2 * th2 * th);
    }
    double P[9], R[9], P2[9], Jso[9];
    hat(phi, P);
    hat(rho, R);
    mat3_mul(P, P, P2);
    for (int i = 0; i < 9; ++i) Jso[i] = ((i % 4 == 0) ? 1.0 : 0.0) + b * P[i] + c1 * P2[i];
    double PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
    mat3_mul(P, R, PR);
    mat3_mul(R, P, RP);
    mat3_mul(PR, P, PRP);
    mat3_mul(P, PR, PPR);
    mat3_mul(RP, P, RPP);
    mat3_mul(PRP, P, PRPP);
    mat3_mul(P, PRP, PPRP);
    double Q[9];
    for (int i = 0; i < 9; ++i)
        Q[i] = 0.5 * R[i] + c1 * (PR[i] + RP[i] + PRP[i]) + c2 * (PPR[i] + RPP[i] - 3.0 * PRP[i]) +
               c3 * (PRPP[i] + PPRP[i]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            J[r * 6 + c] = Jso[r * 3 + c];
            J[r * 6 + 3 + c] = 0.0;
            J[(3 + r) * 6 + c] = Q[r * 3 + c];
            J[(3 + r) * 6 + 3 + c] = Jso[r * 3 + c];
        }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw, "Parallel      */
/* random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64   */
/* multiplies with the key bumped by two Weyl constants between rounds.      */
/* ------------------------------------------------------------------------ */

void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c[0];
        uint64_t p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k[0] += W0; k[1] += W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

#define ORA_TAG_NORMAL 0x4E4F524Du  /* counter word 3 for motion noise */
#define ORA_TAG_RESAMPLE 0x52534D50u /* counter word 3 for the resampling offset */

/* uniform in (0,1) from the top 23 bits: (k + 1/2) 2^-23 is exact in float and double */
static double u23(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

void ora_normal6(uint64_t seed, uint32_t i, uint32_t t, double z[6]) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t a[4], b[4];
    uint32_t c0[4] = {i, t, 0u, ORA_TAG_NORMAL};
    uint32_t c1[4] = {i, t, 1u, ORA_TAG_NORMAL};
    ora_philox4x32_10(c0, key, a);
    ora_philox4x32_10(c1, key, b);
    uint32_t x[6] = {a[0], a[1], a[2], a[3], b[0], b[1]};
    for (int pair = 0; pair < 3; ++pair) {
        double u1 = u23(x[2 * pair]), u2 = u23(x[2 * pair + 1]);
        double r = sqrt(-2.0 * log(u1));
        z[2 * pair] = r * cos(2.0 * M_PI * u2);
        z[2 * pair + 1] = r * sin(2.0 * M_PI * u2);
    }
}

double ora_systematic_u(uint64_t seed, uint32_t t) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c[4] = {0xFFFFFFFFu, t, 0u, ORA_TAG_RESAMPLE}, o[4];
    ora_philox4x32_10(c, key, o);
    double hi = (double)(o[0] >> 5), lo = (double)(o[1] >> 6);
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* likelihood tables                                                         */
/* ------------------------------------------------------------------------ */

static size_t vidx(const ora_grid* g, int ix, int iy, int iz) {
    return ((size_t)iz * (size_t)g->n[1] + (size_t)iy) * (size_t)g->n[0] + (size_t)ix;
}

static double field_value(double d2, double sigma, double r_t) {
    return (d2 <= r_t * r_t) ? exp(-d2 / (2.0 * sigma * sigma)) : 0.0;
}

void ora_build_table(const float* pts, int n, const ora_grid* g, double sigma, double r_t, double* vals) {
    size_t nv = (size_t)g->n[0] * g->n[1] * g->n[2];
    double* d2 = (double*)malloc(nv * sizeof(double));
    for (size_t v = 0; v < nv; ++v) d2[v] = INFINITY;
    for (int j = 0; j < n; ++j) {
        double p[3] = {pts[3 * j], pts[3 * j + 1], pts[3 * j + 2]};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)ceil((p[a] - r_t - g->origin[a]) / g->h);
            hi[a] = (int)floor((p[a] + r_t - g->origin[a]) / g->h);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > g->n[a] - 1) hi[a] = g->n[a] - 1;
        }
        for (int iz = lo[2]; iz <= hi[2]; ++iz)
            for (int iy = lo[1]; iy <= hi[1]; ++iy)
                for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                    double x = g->origin[0] + g->h * ix - p[0];
                    double y = g->origin[1] + g->h * iy - p[1];
                    double z = g->origin[2] + g->h * iz - p[2];
                    double dd = x * x + y * y + z * z;
                    size_t v = vidx(g, ix, iy, iz);
                    if (dd < d2[v]) d2[v] = dd;
                }
    }
    for (size_t v = 0; v < nv; ++v) vals[v] = field_value(d2[v], sigma, r_t);
    free(d2);
}

void ora_build_table_brute(const float* pts, int n, const ora_grid* g, double sigma, double r_t, double* vals) {
    for (int iz = 0; iz < g->n[2]; ++iz)
        for (int iy = 0; iy < g->n[1]; ++iy)
            for (int ix = 0; ix < g->n[0]; ++ix) {
                double best = INFINITY;
                for (int j = 0; j < n; ++j) {
                    double x = g->origin[0] + g->h * ix - (double)pts[3 * j];
                    double y = g->origin[1] + g->h * iy - (double)pts[3 * j + 1];
                    double z = g->origin[2] + g->h * iz - (double)pts[3 * j + 2];
                    double dd = x * x + y * y + z * z;
                    if (dd < best) best = dd;
                }
                vals[vidx(g, ix, iy, iz)] = field_value(best, sigma, r_t);
            }
}

/* Round v >= 0 to a float format with `mant` significant bits whose smallest
 * normal exponent is emin (values below 2^emin use the fixed subnormal step). */
static double round_format(double v, int mant, int emin) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(fabs(v), &e);           /* |v| = f 2^e, f in [0.5, 1) */
    int ex = e - 1;               /* |v| in [2^ex, 2^(ex+1)) */
    if (ex < emin) ex = emin;
    double q = ldexp(1.0, ex - (mant - 1));
    return nearbyint(v / q) * q;  /* default rounding mode: nearest-even */
}

void ora_quantize(const double* in, size_t n, int dtype, double* out) {
    for (size_t i = 0; i < n; ++i) {
        if (dtype == 1) out[i] = round_format(in[i], 8, -126);
        else if (dtype == 2) out[i] = round_format(in[i], 11, -14);
        else out[i] = in[i];
    }
}

int ora_cell_eval(const double* vals, const ora_grid* g, const int c[3], const double u[3],
                  double* L, double dLdu[3]) {
    *L = 0.0;
    dLdu[0] = dLdu[1] = dLdu[2] = 0.0;
    for (int a = 0; a < 3; ++a)
        if (c[a] < 0 || c[a] > g->n[a] - 2) return 0;
    double f[3] = {u[0] - c[0], u[1] - c[1], u[2] - c[2]};
    if (g->coef) {
        const size_t cell = ((size_t)c[2] * (g->n[1] - 1) + c[1]) * (size_t)(g->n[0] - 1) + c[0];
        const double* k = vals + 8 * cell;
        const double x = f[0], y = f[1], z = f[2];
        *L = k[0] + k[1] * x + k[2] * y + k[3] * z + k[4] * x * y + k[5] * x * z + k[6] * y * z + k[7] * x * y * z;
        dLdu[0] = k[1] + k[4] * y + k[5] * z + k[7] * y * z;
        dLdu[1] = k[2] + k[4] * x + k[6] * z + k[7] * x * z;
        dLdu[2] = k[3] + k[5] * x + k[6] * y + k[7] * x * y;
        return 1;
    }
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double v = vals[vidx(g, c[0] + dx, c[1] + dy, c[2] + dz)];
                double wx = dx ? f[0] : 1.0 - f[0];
                double wy = dy ? f[1] : 1.0 - f[1];
                double wz = dz ? f[2] : 1.0 - f[2];
                double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
                *L += v * wx * wy * wz;
                dLdu[0] += v * sx * wy * wz;
                dLdu[1] += v * wx * sy * wz;
                dLdu[2] += v * wx * wy * sz;
            }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* per-particle evaluation                                                   */
/* ------------------------------------------------------------------------ */

/* d l / d xi of one lookup: with R the relative rotation, q = R^T grad_x l and
 * the right perturbation of the current pose moving a scan point p by
 * R(omega x p + v), the derivative is [p x q; q]. */
static void lookup_grad(const double Rrel[9], const double p[3], double h, double L, const double dLdu[3],
                        double eps, double gj[6]) {
    double inv = 1.0 / (L + eps);
    double gx[3] = {dLdu[0] / h * inv, dLdu[1] / h * inv, dLdu[2] / h * inv};
    double q[3];
    for (int r = 0; r < 3; ++r) q[r] = Rrel[0 * 3 + r] * gx[0] + Rrel[1 * 3 + r] * gx[1] + Rrel[2 * 3 + r] * gx[2];
    gj[0] = p[1] * q[2] - p[2] * q[1];
    gj[1] = p[2] * q[0] - p[0] * q[2];
    gj[2] = p[0] * q[1] - p[1] * q[0];
    gj[3] = q[0]; gj[4] = q[1]; gj[5] = q[2];
}

void ora_eval_particle(const double Tt[12], int n_nb, const double* Tk, const double* const* tables,
                       const ora_grid* grids, const float* scan, int N, const ora_eval_params* prm,
                       double* ll, double g[6], double mom[10], double* slack, double* gabs,
                       int* cells, int frozen) {
    double acc_ll = 0.0, acc_g[6] = {0}, acc_m[10] = {0}, acc_s = 0.0, acc_a = 0.0;
    for (int s = 0; s < n_nb; ++s) {
        /* relative pose kT_t = (T_k)^-1 T_t (Eq. 4) */
        double inv[12], rel[12];
        ora_pose_inv(Tk + 12 * s, inv);
        ora_pose_mul(inv, Tt, rel);
        double Rrel[9] = {rel[0], rel[1], rel[2], rel[4], rel[5], rel[6], rel[8], rel[9], rel[10]};
        const ora_grid* gr = &grids[s];
        const double* tab = tables[s];
        for (int j = 0; j < N; ++j) {
            double p[3] = {scan[3 * j], scan[3 * j + 1], scan[3 * j + 2]};
            double x[3], u[3];
            for (int r = 0; r < 3; ++r) {
                x[r] = rel[r * 4 + 0] * p[0] + rel[r * 4 + 1] * p[1] + rel[r * 4 + 2] * p[2] + rel[r * 4 + 3];
                u[r] = (x[r] - gr->origin[r]) / gr->h;
            }
            int c[3];
            int* cslot = cells ? cells + 3 * ((size_t)s * N + j) : NULL;
            if (frozen) {
                c[0] = cslot[0]; c[1] = cslot[1]; c[2] = cslot[2];
            } else {
                for (int a = 0; a < 3; ++a) c[a] = (int)floor(u[a]);
            }
            double L, dL[3];
            int valid = (frozen && c[0] == -1 && c[1] == -1 && c[2] == -1) ? 0 : ora_cell_eval(tab, gr, c, u, &L, dL);
            if (!valid) { L = 0.0; dL[0] = dL[1] = dL[2] = 0.0; }
            if (!frozen && cslot) {
                if (valid) { cslot[0] = c[0]; cslot[1] = c[1]; cslot[2] = c[2]; }
                else { cslot[0] = cslot[1] = cslot[2] = -1; }
            }
            acc_ll += log(L + prm->eps);
            double gj[6];
            lookup_grad(Rrel, p, gr->h, L, dL, prm->eps, gj);
            for (int d = 0; d < 6; ++d) acc_g[d] += gj[d];
            acc_a += sqrt(gj[0] * gj[0] + gj[1] * gj[1] + gj[2] * gj[2] + gj[3] * gj[3] + gj[4] * gj[4] + gj[5] * gj[5]);
            double w = L / (L + prm->eps);
            acc_m[0] += w;
            acc_m[1] += w * p[0]; acc_m[2] += w * p[1]; acc_m[3] += w * p[2];
            acc_m[4] += w * p[0] * p[0]; acc_m[5] += w * p[0] * p[1]; acc_m[6] += w * p[0] * p[2];
            acc_m[7] += w * p[1] * p[1]; acc_m[8] += w * p[1] * p[2]; acc_m[9] += w * p[2] * p[2];
            /* face slack: the other cells a slightly different rounding of u could pick */
            if (!frozen && slack && valid) {
                int near[3], dir[3], nn = 0;
                for (int a = 0; a < 3; ++a) {
                    double f = u[a] - c[a];
                    if (f < prm->face_delta) { near[nn] = a; dir[nn] = -1; ++nn; }
                    else if (1.0 - f < prm->face_delta) { near[nn] = a; dir[nn] = +1; ++nn; }
                }
                for (int mask = 1; mask < (1 << nn); ++mask) {
                    int c2[3] = {c[0], c[1], c[2]};
                    for (int b = 0; b < nn; ++b)
                        if (mask & (1 << b)) c2[near[b]] += dir[b];
                    double L2, dL2[3], g2[6];
                    if (!ora_cell_eval(tab, gr, c2, u, &L2, dL2)) { L2 = 0.0; dL2[0] = dL2[1] = dL2[2] = 0.0; }
                    lookup_grad(Rrel, p, gr->h, L2, dL2, prm->eps, g2);
                    double dd = 0.0;
                    for (int d = 0; d < 6; ++d) dd += (g2[d] - gj[d]) * (g2[d] - gj[d]);
                    acc_s += sqrt(dd);
                }
            }
        }
    }
    if (ll) *ll = acc_ll;
    if (g) for (int d = 0; d < 6; ++d) g[d] = acc_g[d];
    if (mom) for (int d = 0; d < 10; ++d) mom[d] = acc_m[d];
    if (slack) *slack = acc_s;
    if (gabs) *gabs = acc_a;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Newton move, Eq. 5-7                                               */
/* ------------------------------------------------------------------------ */

/* sigma^-2 sum w B^T B with B = [-[p]x | I]:
 *   rotation block  tr(Q) I - Q,  cross block [S]x,  translation block W I. */
void ora_h_from_moments(const double mom[10], double sigma, double H[36]) {
    double W = mom[0];
    double S[3] = {mom[1], mom[2], mom[3]};
    double Q[9] = {mom[4], mom[5], mom[6], mom[5], mom[7], mom[8], mom[6], mom[8], mom[9]};
    double trQ = Q[0] + Q[4] + Q[8];
    double Sx[9];
    hat(S, Sx);
    double k = 1.0 / (sigma * sigma);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            H[r * 6 + c] = k * ((r == c ? trQ : 0.0) - Q[r * 3 + c]);
            H[r * 6 + 3 + c] = k * Sx[r * 3 + c];
            H[(3 + r) * 6 + c] = k * Sx[c * 3 + r];
            H[(3 + r) * 6 + 3 + c] = k * (r == c ? W : 0.0);
        }
}

void ora_h_explicit(const float* scan, int N, const double* w, double sigma, double H[36]) {
    for (int i = 0; i < 36; ++i) H[i] = 0.0;
    for (int j = 0; j < N; ++j) {
        double p[3] = {scan[3 * j], scan[3 * j + 1], scan[3 * j + 2]};
        double P[9], B[18];
        hat(p, P);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                B[r * 6 + c] = -P[r * 3 + c];
                B[r * 6 + 3 + c] = (r == c) ? 1.0 : 0.0;
            }
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b) {
                double s = 0.0;
                for (int r = 0; r < 3; ++r) s += B[r * 6 + a] * B[r * 6 + b];
                H[a * 6 + b] += w[j] * s / (sigma * sigma);
            }
    }
}

/* Cholesky A = L L^T of an n x n matrix; 0 on success, -1 on a non-positive pivot. */
static int cholesky(const double* A, int n, double* L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return -1;
        L[j * n + j] = sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / L[j * n + j];
        }
    }
    return 0;
}

/* psi = (H + lambda diag H)^-1 g by Cholesky, then the clamps (psi = 0 when the
 * damped matrix is not positive definite). H is modified. */
static void damped_step(double H[36], const double g[6], const ora_move_params* mp, double psi[6]) {
    double L[36];
    for (int d = 0; d < 6; ++d) H[d * 6 + d] *= (1.0 + mp->lambda);
    if (cholesky(H, 6, L) != 0) return;
    double y[6];
    for (int i = 0; i < 6; ++i) {        /* L y = g */
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= L[i * 6 + k] * y[k];
        y[i] = s / L[i * 6 + i];
    }
    for (int i = 5; i >= 0; --i) {       /* L^T psi = y */
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k * 6 + i] * psi[k];
        psi[i] = s / L[i * 6 + i];
    }
    double nw = sqrt(psi[0] * psi[0] + psi[1] * psi[1] + psi[2] * psi[2]);
    double nv = sqrt(psi[3] * psi[3] + psi[4] * psi[4] + psi[5] * psi[5]);
    if (nw > mp->theta_max) for (int d = 0; d < 3; ++d) psi[d] *= mp->theta_max / nw;
    if (nv > mp->t_max) for (int d = 3; d < 6; ++d) psi[d] *= mp->t_max / nv;
}

void ora_move(const double Tt[12], const double g[6], const double mom[10], const ora_move_params* mp,
              double Tout[12], double psi[6]) {
    for (int d = 0; d < 6; ++d) psi[d] = 0.0;
    if (mom[0] >= mp->w_min) {
        double H[36];
        ora_h_from_moments(mom, mp->sigma, H);
        damped_step(H, g, mp, psi);
    }
    double E[12];
    ora_se3_exp(psi, E);
    ora_pose_mul(Tt, E, Tout);
}

void ora_move_h(const double Tt[12], const double b[6], const double H[36], const ora_move_params* mp,
                double Tout[12], double psi[6]) {
    for (int d = 0; d < 6; ++d) psi[d] = 0.0;
    double Hc[36];
    memcpy(Hc, H, sizeof(Hc));
    damped_step(Hc, b, mp, psi);
    double E[12];
    ora_se3_exp(psi, E);
    ora_pose_mul(Tt, E, Tout);
}

/* ------------------------------------------------------------------------ */
/* GICP distribution-to-distribution likelihood, Eq. 2-6                     */
/* ------------------------------------------------------------------------ */

/* Inverse of a 3x3 matrix by cofactors; 0 when singular. */
static int inv3(const double A[9], double B[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(fabs(det) > 0.0)) return 0;
    B[0] = c00 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return 1;
}

/* One correspondence: voxel record vox (mean, count, covariance), scan point mu
 * with covariance S (6), relative pose rel. Writes d2 = e^T Omega e and the
 * term's b and H; returns 0 (and zeros) when there is no distribution. */
static int gicp_dist(const double* vox, const double rel[12], const double mu[3], const double* S,
                     double* d2out, double bj[6], double Hj[36]) {
    *d2out = 0.0;
    for (int d = 0; d < 6; ++d) bj[d] = 0.0;
    for (int d = 0; d < 36; ++d) Hj[d] = 0.0;
    if (!vox || !(vox[3] > 0.0)) return 0;
    double R[9] = {rel[0], rel[1], rel[2], rel[4], rel[5], rel[6], rel[8], rel[9], rel[10]};
    double x[3], e[3];
    for (int r = 0; r < 3; ++r) {
        x[r] = R[r * 3] * mu[0] + R[r * 3 + 1] * mu[1] + R[r * 3 + 2] * mu[2] + rel[r * 4 + 3];
        e[r] = vox[r] - x[r];                       /* e = mu' - kT_t mu  (Eq. 4) */
    }
    double Sj[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    double Sv[9] = {vox[4], vox[5], vox[6], vox[5], vox[7], vox[8], vox[6], vox[8], vox[9]};
    double RS[9], C[9], Om[9];
    mat3_mul(R, Sj, RS);
    for (int r = 0; r < 3; ++r)                      /* Sigma' + R Sigma R^T */
        for (int c = 0; c < 3; ++c)
            C[r * 3 + c] = Sv[r * 3 + c] + RS[r * 3] * R[c * 3] + RS[r * 3 + 1] * R[c * 3 + 1] + RS[r * 3 + 2] * R[c * 3 + 2];
    if (!inv3(C, Om)) return 0;
    double Oe[3];
    for (int r = 0; r < 3; ++r) Oe[r] = Om[r * 3] * e[0] + Om[r * 3 + 1] * e[1] + Om[r * 3 + 2] * e[2];
    *d2out = e[0] * Oe[0] + e[1] * Oe[1] + e[2] * Oe[2];     /* Eq. 3: the term is -d2 */
    /* J = d(kT_t exp(xi) mu)/d xi = R [-[mu]x | I]  (3 x 6) */
    double M[9], J[18];
    hat(mu, M);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            J[r * 6 + c] = -(R[r * 3] * M[c] + R[r * 3 + 1] * M[3 + c] + R[r * 3 + 2] * M[6 + c]);
            J[r * 6 + 3 + c] = R[r * 3 + c];
        }
    for (int a = 0; a < 6; ++a) {                   /* b = J^T Omega e, H = J^T Omega J (Eq. 6) */
        bj[a] = J[a] * Oe[0] + J[6 + a] * Oe[1] + J[12 + a] * Oe[2];
        double OJ[3];
        for (int r = 0; r < 3; ++r) OJ[r] = Om[r * 3] * J[a] + Om[r * 3 + 1] * J[6 + a] + Om[r * 3 + 2] * J[12 + a];
        for (int c = 0; c < 6; ++c) Hj[c * 6 + a] = J[c] * OJ[0] + J[6 + c] * OJ[1] + J[12 + c] * OJ[2];
    }
    return 1;
}

/* The capped term: an inlier (a distribution and d2 < tau) adds -d2, b, H;
 * anything else adds -tau and no gradient. Returns 1 for an inlier. */
static int gicp_term(const double* vox, const double rel[12], const double mu[3], const double* S, double tau,
                     double* l, double bj[6], double Hj[36], double* d2, int* has) {
    *has = gicp_dist(vox, rel, mu, S, d2, bj, Hj);
    if (*has && *d2 < tau) {
        *l = -*d2;
        return 1;
    }
    *l = -tau;
    for (int d = 0; d < 6; ++d) bj[d] = 0.0;
    for (int d = 0; d < 36; ++d) Hj[d] = 0.0;
    return 0;
}

void ora_gicp_eval_particle(const double Tt[12], int n_nb, const double* Tk, const double* const* maps,
                            const ora_grid* grids, const float* scan, const double* scov, int N, double tau,
                            double face_delta, double gate_delta, double* ll, double b[6], double H[36],
                            double slack[3], int* nvalid) {
    double acc_l = 0.0, acc_b[6] = {0}, acc_H[36] = {0}, sl[3] = {0, 0, 0};
    int nv = 0;
    for (int s = 0; s < n_nb; ++s) {
        double inv[12], rel[12];
        ora_pose_inv(Tk + 12 * s, inv);
        ora_pose_mul(inv, Tt, rel);                 /* kT_t = (T_k)^-1 T_t */
        const ora_grid* g = &grids[s];
        const double* map = maps[s];
        for (int j = 0; j < N; ++j) {
            double mu[3] = {scan[3 * j], scan[3 * j + 1], scan[3 * j + 2]};
            double u[3];
            int c[3], inside = 1;
            for (int r = 0; r < 3; ++r) {
                double x = rel[r * 4] * mu[0] + rel[r * 4 + 1] * mu[1] + rel[r * 4 + 2] * mu[2] + rel[r * 4 + 3];
                u[r] = (x - g->origin[r]) / g->h;
                c[r] = (int)floor(u[r]);
                if (c[r] < 0 || c[r] >= g->n[r]) inside = 0;
            }
            double l, bj[6], Hj[36], d2;
            int has;
            int ok = gicp_term(inside ? map + 10 * vidx(g, c[0], c[1], c[2]) : NULL, rel, mu, scov + 6 * (size_t)j,
                               tau, &l, bj, Hj, &d2, &has);
            nv += ok;
            if (slack && has && fabs(d2 - tau) < gate_delta * tau) {
                /* at the cap, a different rounding of d2 flips the term in or out */
                double bg[6], Hg[36], dd;
                gicp_dist(map + 10 * vidx(g, c[0], c[1], c[2]), rel, mu, scov + 6 * (size_t)j, &dd, bg, Hg);
                double nb = 0.0, nH = 0.0;
                for (int d = 0; d < 6; ++d) nb += bg[d] * bg[d];
                for (int d = 0; d < 36; ++d) nH += Hg[d] * Hg[d];
                sl[0] += fabs(dd - tau);
                sl[1] += sqrt(nb);
                sl[2] += sqrt(nH);
            }
            acc_l += l;
            for (int d = 0; d < 6; ++d) acc_b[d] += bj[d];
            for (int d = 0; d < 36; ++d) acc_H[d] += Hj[d];
            if (slack) {
                /* the voxel across the nearest face, when u is within face_delta of it */
                int ax = -1, dir = 0;
                double best = face_delta;
                for (int r = 0; r < 3; ++r) {
                    double f = u[r] - floor(u[r]);
                    if (f < best) { best = f; ax = r; dir = -1; }
                    if (1.0 - f < best) { best = 1.0 - f; ax = r; dir = +1; }
                }
                if (ax >= 0) {
                    int c2[3] = {c[0], c[1], c[2]};
                    c2[ax] += dir;
                    int in2 = 1;
                    for (int r = 0; r < 3; ++r)
                        if (c2[r] < 0 || c2[r] >= g->n[r]) in2 = 0;
                    double l2, b2[6], H2[36], dd2;
                    int has2;
                    gicp_term(in2 ? map + 10 * vidx(g, c2[0], c2[1], c2[2]) : NULL, rel, mu, scov + 6 * (size_t)j,
                              tau, &l2, b2, H2, &dd2, &has2);
                    double db = 0.0, dH = 0.0;
                    for (int d = 0; d < 6; ++d) db += (b2[d] - bj[d]) * (b2[d] - bj[d]);
                    for (int d = 0; d < 36; ++d) dH += (H2[d] - Hj[d]) * (H2[d] - Hj[d]);
                    sl[0] += fabs(l2 - l);
                    sl[1] += sqrt(db);
                    sl[2] += sqrt(dH);
                }
            }
        }
    }
    if (ll) *ll = acc_l;
    if (b) for (int d = 0; d < 6; ++d) b[d] = acc_b[d];
    if (H) for (int d = 0; d < 36; ++d) H[d] = acc_H[d];
    if (slack) for (int d = 0; d < 3; ++d) slack[d] = sl[d];
    if (nvalid) *nvalid = nv;
}

/* ------------------------------------------------------------------------ */
/* keyframe pose propagation, Eq. 8-10                                        */
/* ------------------------------------------------------------------------ */

void ora_propagate(const double psi[6], const int* nbr, int k_nb, int K, const double* D, double Dt, double* kf_i) {
    int o = -1;
    for (int s = 0; s < k_nb; ++s)
        if (nbr[s] >= 0 && (o < 0 || nbr[s] < o)) o = nbr[s];
    if (o < 0) return;
    double total = Dt - D[o];           /* d(t_t, t_o) */
    if (!(total > 0.0)) return;
    for (int k = o + 1; k < K; ++k) {
        double r = (D[k] - D[o]) / total;   /* d(t_k, t_o) / d(t_t, t_o) */
        if (r < 0.0) r = 0.0;
        if (r > 1.0) r = 1.0;
        double pk[6], E[12];
        for (int d = 0; d < 6; ++d) pk[d] = r * psi[d];
        ora_se3_exp(pk, E);
        ora_pose_mul(kf_i + 12 * (size_t)k, E, kf_i + 12 * (size_t)k);
    }
}

int ora_loop(const int* nbr, int k_nb, int K, int recent) {
    if (recent <= 0) return 1;
    int o = -1;
    for (int s = 0; s < k_nb; ++s)
        if (nbr[s] >= 0 && (o < 0 || nbr[s] < o)) o = nbr[s];
    return o >= 0 && o < K - recent;
}

/* ------------------------------------------------------------------------ */
/* neighbours, prediction                                                    */
/* ------------------------------------------------------------------------ */

void ora_select_nbrs(const double Tt[12], const double* kf_t, int K, int k_nb, int* idx) {
    float tx = (float)Tt[3], ty = (float)Tt[7], tz = (float)Tt[11];
    float* d2 = (float*)malloc(sizeof(float) * (K > 0 ? K : 1));
    char* used = (char*)calloc(K > 0 ? K : 1, 1);
    for (int k = 0; k < K; ++k) {
        float dx = (float)kf_t[3 * k] - tx;
        float dy = (float)kf_t[3 * k + 1] - ty;
        float dz = (float)kf_t[3 * k + 2] - tz;
        float xx = dx * dx, yy = dy * dy, zz = dz * dz;
        float s = xx + yy;
        d2[k] = s + zz;
    }
    for (int s = 0; s < k_nb; ++s) {
        int best = -1;
        for (int k = 0; k < K; ++k) {
            if (used[k]) continue;
            if (best < 0 || d2[k] < d2[best]) best = k;
        }
        idx[s] = best;
        if (best >= 0) used[best] = 1;
    }
    free(d2);
    free(used);
}

/* Cholesky of a positive semi-definite matrix: a zero pivot zeroes its column. */
static void cholesky_psd(const double* A, int n, double* L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) continue;
        L[j * n + j] = sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / L[j * n + j];
        }
    }
}

void ora_predict(const double T[12], const double dT[12], const double cov[36], const double z[6],
                 double Tout[12]) {
    double Lc[36], delta[6], E[12], TdT[12];
    cholesky_psd(cov, 6, Lc);
    for (int r = 0; r < 6; ++r) {
        double s = 0.0;
        for (int c = 0; c <= r; ++c) s += Lc[r * 6 + c] * z[c];
        delta[r] = s;
    }
    ora_se3_exp(delta, E);
    ora_pose_mul(T, dT, TdT);
    ora_pose_mul(TdT, E, Tout);
}

/* ------------------------------------------------------------------------ */
/* weights and resampling                                                    */
/* ------------------------------------------------------------------------ */

void ora_lse(const double* logw, const double* ll, int P, double* logw_out, double* w,
             double* M, double* logS, int* argmax, double* ess) {
    double m = -INFINITY;
    int am = 0;
    for (int i = 0; i < P; ++i) {
        double v = logw[i] + ll[i];
        logw_out[i] = v;
        if (v > m) { m = v; am = i; }
    }
    double S = 0.0;
    for (int i = 0; i < P; ++i) S += exp(logw_out[i] - m);
    double ls = log(S);
    double s2 = 0.0;
    for (int i = 0; i < P; ++i) {
        w[i] = exp(logw_out[i] - m - ls);
        s2 += w[i] * w[i];
    }
    *M = m;
    *logS = ls;
    *argmax = am;
    *ess = 1.0 / s2;
}

void ora_resample(const double* w, int P, double u, int* anc) {
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
    uint64_t run = 0;
    for (int i = 0; i < P; ++i) {
        double q = nearbyint(w[i] * 4503599627370496.0);   /* w on the 2^-52 grid */
        run += (uint64_t)q;
        C[i] = run;
    }
    double Sq = (double)run;
    int i = 0;
    for (int m = 0; m < P; ++m) {
        double t1 = u + (double)m;
        double t2 = t1 / (double)P;
        double tau = t2 * Sq;
        while (i < P && !((double)C[i] > tau)) ++i;
        anc[m] = (i < P) ? i : P - 1;
        if (i >= P) i = P - 1;
    }
    free(C);
}

int ora_prune(const double* x, const double* w, const double* ll, int P, int argmax, double prune_w,
              double ll_cut, double u, int* anc, double* logw_out) {
    /* 1. the dead set */
    double ll_max = -INFINITY;
    if (ll)
        for (int i = 0; i < P; ++i)
            if (ll[i] > ll_max) ll_max = ll[i];
    int* dead = (int*)malloc(sizeof(int) * (P > 0 ? P : 1));
    int D = 0;
    for (int i = 0; i < P; ++i) {
        int d = !(w[i] >= prune_w);
        if (ll && ll_cut > -INFINITY && !(ll[i] - ll_max >= ll_cut)) d = 1;
        if (i == argmax) d = 0;
        dead[i] = d;
        D += d;
    }
    /* 2. cumulative quantised weights of the survivors */
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
    uint64_t run = 0;
    for (int i = 0; i < P; ++i) {
        if (!dead[i] && w[i] > 0.0 && w[i] <= 1.0) run += (uint64_t)nearbyint(w[i] * 4503599627370496.0);
        C[i] = run;
    }
    double S = (double)run;
    /* 3. one systematic comb of D teeth over the survivors */
    int* copies = (int*)calloc(P > 0 ? P : 1, sizeof(int));
    for (int i = 0; i < P; ++i) anc[i] = i;
    int r = 0;
    for (int i = 0; i < P && S > 0.0; ++i) {
        if (!dead[i]) continue;
        double tau = ((u + (double)r) / (double)D) * S;
        if (tau > S - 1.0) tau = S - 1.0;
        int a = 0;
        while (!((double)C[a] > tau)) ++a;
        anc[i] = a;
        copies[a] += 1;
        ++r;
    }
    /* 4. weights: each survivor's weight split evenly over it and its copies */
    for (int i = 0; i < P; ++i) {
        int a = anc[i];
        logw_out[i] = copies[a] ? x[a] - log1p((double)copies[a]) : x[a];
    }
    free(dead); free(C); free(copies);
    return D;
}

/* ------------------------------------------------------------------------ */
/* keyframe insertion by overlap, Sec. III-E                                 */
/* ------------------------------------------------------------------------ */

void ora_occupancy_grid(const float* pts, int n, double h, ora_grid* g) {
    for (int a = 0; a < 3; ++a) {
        double mn = INFINITY, mx = -INFINITY;
        for (int i = 0; i < n; ++i) {
            double v = pts[3 * i + a];
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        if (n == 0) mn = mx = 0.0;
        double lo = floor(mn / h) - 1.0, hi = floor(mx / h) + 1.0;
        g->origin[a] = lo * h;
        g->n[a] = (int)(hi - lo) + 1;
    }
    g->h = h;
}

double ora_overlap(const float* kf_pts, int nk, const ora_grid* g, const float* scan, int n, const double T_rel[12]) {
    size_t nv = (size_t)g->n[0] * g->n[1] * g->n[2];
    unsigned char* occ = (unsigned char*)calloc(nv > 0 ? nv : 1, 1);
    for (int i = 0; i < nk; ++i) {
        int c[3], in = 1;
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(((double)kf_pts[3 * i + a] - g->origin[a]) / g->h);
            if (c[a] < 0 || c[a] >= g->n[a]) in = 0;
        }
        if (in) occ[vidx(g, c[0], c[1], c[2])] = 1;
    }
    int hit = 0;
    for (int j = 0; j < n; ++j) {
        double p[3] = {scan[3 * j], scan[3 * j + 1], scan[3 * j + 2]};
        int c[3], in = 1;
        for (int a = 0; a < 3; ++a) {
            double x = T_rel[4 * a] * p[0] + T_rel[4 * a + 1] * p[1];
            x = x + T_rel[4 * a + 2] * p[2];
            x = x + T_rel[4 * a + 3];
            c[a] = (int)floor((x - g->origin[a]) / g->h);
            if (c[a] < 0 || c[a] >= g->n[a]) in = 0;
        }
        if (in && occ[vidx(g, c[0], c[1], c[2])]) ++hit;
    }
    free(occ);
    return n > 0 ? (double)hit / (double)n : 0.0;
}

/* ------------------------------------------------------------------------ */
/* whole frame                                                               */
/* ------------------------------------------------------------------------ */

void ora_step(int P, int K, double* poses, double* kf_poses, double* logw,
              const double* const* tables, const ora_grid* grids,
              const float* scan, const double* scov, int N, const double dT[12], const double cov[36],
              uint32_t frame, const double* z, const double* u, const ora_step_params* sp,
              const double* kf_path, double path_now,
              ora_step_out* out, double* ll_out, double* w_out, int* anc_out, int* nbr_out) {
    int k_nb = sp->k_nb < K ? sp->k_nb : K;
    int* nbr = (int*)malloc(sizeof(int) * (size_t)P * (k_nb > 0 ? k_nb : 1));
    double* ll = (double*)malloc(sizeof(double) * P);
    double* lw = (double*)malloc(sizeof(double) * P);
    double* w = (double*)malloc(sizeof(double) * P);
    ora_eval_params ep = {sp->eps, sp->face_delta};
    ora_move_params mp = {sp->sigma, sp->lambda, sp->theta_max, sp->t_max, sp->w_min};

    /* prediction, Eq. 1 */
    for (int i = 0; i < P; ++i) {
        double zi[6];
        if (z) memcpy(zi, z + 6 * (size_t)i, sizeof(zi));
        else ora_normal6(sp->seed, (uint32_t)i, frame, zi);
        ora_predict(poses + 12 * (size_t)i, dT, cov, zi, poses + 12 * (size_t)i);
    }
    /* neighbour keyframes by translation distance, frozen for the frame */
    double* kt = (double*)malloc(sizeof(double) * 3 * (K > 0 ? K : 1));
    for (int i = 0; i < P; ++i) {
        for (int k = 0; k < K; ++k) {
            const double* Tk = kf_poses + ((size_t)k * P + i) * 12;
            kt[3 * k] = Tk[3]; kt[3 * k + 1] = Tk[7]; kt[3 * k + 2] = Tk[11];
        }
        ora_select_nbrs(poses + 12 * (size_t)i, kt, K, k_nb, nbr + (size_t)i * k_nb);
    }
    free(kt);
    double* Tk = (double*)malloc(sizeof(double) * 12 * (k_nb > 0 ? k_nb : 1));
    const double** tabs = (const double**)malloc(sizeof(double*) * (k_nb > 0 ? k_nb : 1));
    ora_grid* grs = (ora_grid*)malloc(sizeof(ora_grid) * (k_nb > 0 ? k_nb : 1));
    /* gradient-guided moves, Eq. 5-7, then the value pass */
    for (int pass = 0; pass <= sp->steps; ++pass) {
        for (int i = 0; i < P; ++i) {
            for (int s = 0; s < k_nb; ++s) {
                int k = nbr[(size_t)i * k_nb + s];
                memcpy(Tk + 12 * s, kf_poses + ((size_t)k * P + i) * 12, 12 * sizeof(double));
                tabs[s] = tables[k];
                grs[s] = grids[k];
            }
            double g[6], mom[10];
            if (pass < sp->steps) {
                const int* nb = nbr + (size_t)i * k_nb;
                if (!ora_loop(nb, k_nb, K, sp->loop_recent)) continue;   /* Sec. III-C2 */
                double psi[6];
                if (sp->model == 1) {
                    double Hg[36];
                    ora_gicp_eval_particle(poses + 12 * (size_t)i, k_nb, Tk, tabs, grs, scan, scov, N, sp->gicp_tau,
                                           sp->face_delta, 0.0, NULL, g, Hg, NULL, NULL);
                    ora_move_h(poses + 12 * (size_t)i, g, Hg, &mp, poses + 12 * (size_t)i, psi);
                } else {
                    ora_eval_particle(poses + 12 * (size_t)i, k_nb, Tk, tabs, grs, scan, N, &ep,
                                      NULL, g, mom, NULL, NULL, NULL, 0);
                    ora_move(poses + 12 * (size_t)i, g, mom, &mp, poses + 12 * (size_t)i, psi);
                }
                if (sp->propagate && kf_path) {
                    double* kfi = (double*)malloc(sizeof(double) * 12 * (size_t)K);
                    for (int k = 0; k < K; ++k)
                        memcpy(kfi + 12 * (size_t)k, kf_poses + ((size_t)k * P + i) * 12, 12 * sizeof(double));
                    ora_propagate(psi, nb, k_nb, K, kf_path, path_now, kfi);
                    for (int k = 0; k < K; ++k)
                        memcpy(kf_poses + ((size_t)k * P + i) * 12, kfi + 12 * (size_t)k, 12 * sizeof(double));
                    free(kfi);
                }
            } else if (sp->model == 1) {
                ora_gicp_eval_particle(poses + 12 * (size_t)i, k_nb, Tk, tabs, grs, scan, scov, N, sp->gicp_tau,
                                       sp->face_delta, 0.0, ll + i, NULL, NULL, NULL, NULL);
            } else {
                ora_eval_particle(poses + 12 * (size_t)i, k_nb, Tk, tabs, grs, scan, N, &ep,
                                  ll + i, NULL, NULL, NULL, NULL, NULL, 0);
            }
        }
    }
    free(Tk); free(tabs); free(grs);
    /* importance weighting, Eq. 11 */
    double M, logS, ess;
    int am;
    ora_lse(logw, ll, P, lw, w, &M, &logS, &am, &ess);
    memcpy(out->estimate, poses + 12 * (size_t)am, 12 * sizeof(double));
    out->ess = ess;
    out->max_w = w[am];
    out->argmax = am;
    if (ll_out) memcpy(ll_out, ll, sizeof(double) * P);
    if (w_out) memcpy(w_out, w, sizeof(double) * P);
    if (nbr_out) memcpy(nbr_out, nbr, sizeof(int) * (size_t)P * k_nb);
    int do_rs = (sp->resample == 0) || (sp->resample == 1 && ess < 0.5 * P);
    out->resampled = do_rs;
    out->pruned = 0;
    if (sp->resample == 3) {
        /* dead-particle pruning, Sec. III-F: refill dead slots from the survivors */
        int* anc = (int*)malloc(sizeof(int) * P);
        double* x = (double*)malloc(sizeof(double) * P);
        for (int i = 0; i < P; ++i) x[i] = lw[i] - M - logS;
        double uu = u ? *u : ora_systematic_u(sp->seed, frame);
        out->pruned = ora_prune(x, w, ll, P, am, sp->prune_w, sp->ll_cut, uu, anc, logw);
        for (int m = 0; m < P; ++m) {
            if (anc[m] == m) continue;
            memcpy(poses + 12 * (size_t)m, poses + 12 * (size_t)anc[m], 12 * sizeof(double));
            for (int k = 0; k < K; ++k) {
                double* base = kf_poses + (size_t)k * P * 12;
                memcpy(base + 12 * (size_t)m, base + 12 * (size_t)anc[m], 12 * sizeof(double));
            }
        }
        if (anc_out) memcpy(anc_out, anc, sizeof(int) * P);
        free(anc); free(x);
    } else if (do_rs) {
        int* anc = (int*)malloc(sizeof(int) * P);
        double uu = u ? *u : ora_systematic_u(sp->seed, frame);
        ora_resample(w, P, uu, anc);
        double* np = (double*)malloc(sizeof(double) * 12 * (size_t)P);
        for (int m = 0; m < P; ++m) memcpy(np + 12 * (size_t)m, poses + 12 * (size_t)anc[m], 12 * sizeof(double));
        memcpy(poses, np, sizeof(double) * 12 * (size_t)P);
        for (int k = 0; k < K; ++k) {
            double* base = kf_poses + (size_t)k * P * 12;
            for (int m = 0; m < P; ++m) memcpy(np + 12 * (size_t)m, base + 12 * (size_t)anc[m], 12 * sizeof(double));
            memcpy(base, np, sizeof(double) * 12 * (size_t)P);
        }
        free(np);
        for (int m = 0; m < P; ++m) logw[m] = -log((double)P);
        if (anc_out) memcpy(anc_out, anc, sizeof(int) * P);
        free(anc);
    } else {
        for (int i = 0; i < P; ++i) logw[i] = lw[i] - M - logS;
        if (anc_out) for (int i = 0; i < P; ++i) anc_out[i] = i;
    }
    free(nbr); free(ll); free(lw); free(w);
}
