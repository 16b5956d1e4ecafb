/*
 * Oracle for the FMM gravitational force solve of Mukherjee, Zhu, Trac &
 * Rodriguez (2021), "Fast Multipole Methods for N-body Simulations of
 * Collisional Star Systems".
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow CPU implementation
 * that the tests, the smoke check and the benchmark's CPU-baseline leg use to
 * check the GPU library. The GPU library never links, loads or calls it, and
 * the two share no code.
 *
 * Everything is FP64 except the scalar-force estimate f, which the MAC uses
 * only as an estimate (Section 2.3) and which is evaluated in FP32 with a
 * fixed operation order (the paper fixes neither). Compile with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Notation follows Section 2.2 of the paper and the solid harmonics of
 * Dehnen (2014) that it adopts:
 *   Upsilon_n^m(r) = r^n Pbar_n^m(cos t) e^{i m phi} / (n+m)!   (regular)
 *   Theta_n^m(r)   = (n-m)! Pbar_n^m(cos t) e^{i m phi} / r^{n+1} (irregular)
 * with Pbar the associated Legendre function without the Condon-Shortley
 * phase, and X_n^{-m} = (-1)^m conj(X_n^m). Only m >= 0 is stored, at index
 * n(n+1)/2 + m.
 *
 * Steps, each in the paper's order:
 *   octree (Fig. 1, Sec. 2.1) -> P2M (Eq. moments, Sec. 2.2) -> M2M up
 *   -> scalar-force estimate f with theta < 1 (Sec. 2.3)
 *   -> error-controlled dual-tree walk with the MAC of Sec. 2.3
 *   -> M2L on accepted pairs / P2P on leaf pairs (Sec. 2.1)
 *   -> L2L down -> L2P.
 * The M2L here is the plain O(p^4) translation (the definition that the
 * rotation-accelerated form of Sec. 2.4 reproduces exactly), not the rotated
 * form.
 *
 * Plummer softening (Appendix B: phi(r) = -G m / sqrt(r^2 + eps_soft^2)).
 * The paper gives only the kernel; the reading here:
 *  - the direct sum, P2P and the near part of f use the softened kernel;
 *  - the far field stays the multipole expansion of 1/r;
 *  - the MAC adds, on each side, the bound of what that omits: for bodies
 *    at distance d >= d_min = r - r_A - r_B, the softened and Newtonian
 *    accelerations of a body of mass m differ by at most 1.5 m eps_soft^2 /
 *    d^4, so a cell of mass M_A differs by at most 1.5 M_A eps_soft^2 / d_min^4;
 *  - eps_soft = 0 takes none of these branches (the Newtonian solve).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 30
#define ORC_MAXLEVEL 21

typedef struct { double re, im; } cplx;

static double FACT[2 * ORC_MAXP + 4];
static double BINOM[ORC_MAXP + 1][ORC_MAXP + 1];

static void init_tables(void) {
    FACT[0] = 1.0;
    for (int k = 1; k < 2 * ORC_MAXP + 4; ++k) FACT[k] = FACT[k - 1] * (double)k;
    for (int n = 0; n <= ORC_MAXP; ++n) {
        BINOM[n][0] = 1.0;
        BINOM[n][n] = 1.0;
        for (int k = 1; k < n; ++k) BINOM[n][k] = BINOM[n - 1][k - 1] + BINOM[n - 1][k];
    }
}

static inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }
static inline int ncoef(int p) { return (p + 1) * (p + 2) / 2; }

static inline cplx cmul(cplx a, cplx b) {
    cplx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}
static inline cplx cconj(cplx a) { a.im = -a.im; return a; }

/* X_n^m for any m in [-n, n], from the m >= 0 storage. */
static inline cplx getc(const cplx* a, int n, int m) {
    if (m >= 0) return a[tri(n, m)];
    cplx v = a[tri(n, -m)];
    v.im = -v.im;
    if ((-m) & 1) { v.re = -v.re; v.im = -v.im; }
    return v;
}

/* Regular solid harmonics Upsilon_n^m(x,y,z), 0 <= m <= n <= p, by the
 * recurrences of Dehnen (2014) eqs. 52-54, which the paper cites:
 *   U_0^0 = 1, U_m^m = (x+iy) U_{m-1}^{m-1} / (2m), U_{m+1}^m = z U_m^m,
 *   U_n^m = [(2n-1) z U_{n-1}^m - r^2 U_{n-2}^m] / ((n+m)(n-m)).          */
void orc_regular(int p, double x, double y, double z, cplx* out) {
    double r2 = x * x + y * y + z * z;
    out[0].re = 1.0; out[0].im = 0.0;
    cplx xp = {x, y};
    for (int m = 1; m <= p; ++m) {
        cplx v = cmul(xp, out[tri(m - 1, m - 1)]);
        out[tri(m, m)].re = v.re / (double)(2 * m);
        out[tri(m, m)].im = v.im / (double)(2 * m);
    }
    for (int m = 0; m < p; ++m) {
        out[tri(m + 1, m)].re = z * out[tri(m, m)].re;
        out[tri(m + 1, m)].im = z * out[tri(m, m)].im;
    }
    for (int m = 0; m <= p; ++m) {
        for (int n = m + 2; n <= p; ++n) {
            double c = (double)((n + m) * (n - m));
            cplx a = out[tri(n - 1, m)], b = out[tri(n - 2, m)];
            out[tri(n, m)].re = ((double)(2 * n - 1) * z * a.re - r2 * b.re) / c;
            out[tri(n, m)].im = ((double)(2 * n - 1) * z * a.im - r2 * b.im) / c;
        }
    }
}

/* Irregular solid harmonics Theta_n^m(x,y,z):
 *   T_0^0 = 1/r, T_m^m = (2m-1)(x+iy) T_{m-1}^{m-1} / r^2,
 *   T_n^m = [(2n-1) z T_{n-1}^m - ((n-1)^2 - m^2) T_{n-2}^m] / r^2.      */
void orc_irregular(int p, double x, double y, double z, cplx* out) {
    double r2 = x * x + y * y + z * z;
    out[0].re = 1.0 / sqrt(r2); out[0].im = 0.0;
    cplx xp = {x, y};
    for (int m = 1; m <= p; ++m) {
        cplx v = cmul(xp, out[tri(m - 1, m - 1)]);
        out[tri(m, m)].re = (double)(2 * m - 1) * v.re / r2;
        out[tri(m, m)].im = (double)(2 * m - 1) * v.im / r2;
    }
    for (int m = 0; m <= p; ++m) {
        for (int n = m + 1; n <= p; ++n) {
            cplx a = out[tri(n - 1, m)];
            double c1 = (double)(2 * n - 1);
            if (n == m + 1) {
                out[tri(n, m)].re = c1 * z * a.re / r2;
                out[tri(n, m)].im = c1 * z * a.im / r2;
            } else {
                cplx b = out[tri(n - 2, m)];
                double c2 = (double)((n - 1) * (n - 1) - m * m);
                out[tri(n, m)].re = (c1 * z * a.re - c2 * b.re) / r2;
                out[tri(n, m)].im = (c1 * z * a.im - c2 * b.im) / r2;
            }
        }
    }
}

/* ---------------------------------------------------------------- operators */

/* P2M, Eq. (moments): M_n^m += sum_i m_i Upsilon_n^m(x_i - c). */
void orc_p2m(int p, int64_t n, const double* x, const double* y, const double* z,
             const double* m, double cx, double cy, double cz, cplx* M) {
    cplx R[ncoef(ORC_MAXP)];
    for (int64_t i = 0; i < n; ++i) {
        orc_regular(p, x[i] - cx, y[i] - cy, z[i] - cz, R);
        for (int k = 0; k < ncoef(p); ++k) {
            M[k].re += m[i] * R[k].re;
            M[k].im += m[i] * R[k].im;
        }
    }
}

/* M2M: shift a multipole about zc to zp (exact, no truncation):
 * M_n^m(zp) += sum_{k<=n} sum_l Upsilon_k^l(zc - zp) M_{n-k}^{m-l}(zc). */
void orc_m2m(int p, const cplx* Mc, double bx, double by, double bz, cplx* Mp) {
    cplx R[ncoef(ORC_MAXP)];
    orc_regular(p, bx, by, bz, R);
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx s = {0.0, 0.0};
            for (int k = 0; k <= n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int mm = m - l;
                    if (mm > n - k || mm < -(n - k)) continue;
                    cplx t = cmul(getc(R, k, l), getc(Mc, n - k, mm));
                    s.re += t.re; s.im += t.im;
                }
            Mp[tri(n, m)].re += s.re;
            Mp[tri(n, m)].im += s.im;
        }
}

/* M2L: local coefficients about zb from a multipole about za, truncated at
 * total degree p: F_n^m += sum_{k<=p-n} sum_l (-1)^k conj(M_k^l)
 *                                         Theta_{n+k}^{m+l}(za - zb).     */
void orc_m2l(int p, const cplx* M, double rx, double ry, double rz, cplx* F) {
    cplx T[ncoef(ORC_MAXP)];
    orc_irregular(p, rx, ry, rz, T);
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx s = {0.0, 0.0};
            for (int k = 0; k <= p - n; ++k)
                for (int l = -k; l <= k; ++l) {
                    cplx t = cmul(cconj(getc(M, k, l)), getc(T, n + k, m + l));
                    if (k & 1) { t.re = -t.re; t.im = -t.im; }
                    s.re += t.re; s.im += t.im;
                }
            F[tri(n, m)].re += s.re;
            F[tri(n, m)].im += s.im;
        }
}

/* L2L: shift local coefficients about zp to zc (exact for degree <= p):
 * F_n^m(zc) += sum_{k<=p-n} sum_l conj(Upsilon_k^l(zc - zp)) F_{n+k}^{m+l}(zp). */
void orc_l2l(int p, const cplx* Fp, double bx, double by, double bz, cplx* Fc) {
    cplx R[ncoef(ORC_MAXP)];
    orc_regular(p, bx, by, bz, R);
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx s = {0.0, 0.0};
            for (int k = 0; k <= p - n; ++k)
                for (int l = -k; l <= k; ++l) {
                    cplx t = cmul(cconj(getc(R, k, l)), getc(Fp, n + k, m + l));
                    s.re += t.re; s.im += t.im;
                }
            Fc[tri(n, m)].re += s.re;
            Fc[tri(n, m)].im += s.im;
        }
}

/* L2P: potential phi = -sum_{n,m} conj(Upsilon_n^m(d)) F_n^m and
 * acceleration a = (Re F_1^1, Im F_1^1, F_1^0) evaluated at d (without G):
 * the degree-1 local coefficients at the particle are the gradient of -phi. */
void orc_l2p(int p, const cplx* F, double dx, double dy, double dz,
             double* phi, double* ax, double* ay, double* az) {
    cplx R[ncoef(ORC_MAXP)];
    orc_regular(p, dx, dy, dz, R);
    double s = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx t = cmul(cconj(getc(R, n, m)), getc(F, n, m));
            s += t.re;
        }
    cplx f10 = {0.0, 0.0}, f11 = {0.0, 0.0};
    for (int k = 0; k <= p - 1; ++k)
        for (int l = -k; l <= k; ++l) {
            cplx r = cconj(getc(R, k, l));
            cplx t0 = cmul(r, getc(F, 1 + k, l));
            f10.re += t0.re; f10.im += t0.im;
            if (1 + l <= 1 + k) {
                cplx t1 = cmul(r, getc(F, 1 + k, 1 + l));
                f11.re += t1.re; f11.im += t1.im;
            }
        }
    *phi = -s;
    *ax = f11.re;
    *ay = f11.im;
    *az = f10.re;
}

/* Potential of a multipole about c at a point x (far field):
 * phi = -sum_{n,m} conj(M_n^m) Theta_n^m(x - c), without G. */
double orc_eval_multipole(int p, const cplx* M, double cx, double cy, double cz,
                          double x, double y, double z) {
    cplx T[ncoef(ORC_MAXP)];
    orc_irregular(p, x - cx, y - cy, z - cz, T);
    double s = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) s += cmul(cconj(getc(M, n, m)), getc(T, n, m)).re;
    return -s;
}

/* ---------------------------------------------------------- derivatives */

/* Derivative c (0: x, 1: y, 2: z) of a family X_n^m that obeys the ladder
 * relations of the regular harmonics, with d+ = dx + i dy, d- = dx - i dy:
 *   dz X_n^m = X_{n-1}^m,  d+ X_n^m = -X_{n-1}^{m+1},  d- X_n^m = X_{n-1}^{m-1}
 * (they follow from the recurrences above; the pins check them against
 * finite differences). So
 *   dx X_n^m = (X_{n-1}^{m-1} - X_{n-1}^{m+1}) / 2
 *   dy X_n^m = i (X_{n-1}^{m+1} + X_{n-1}^{m-1}) / 2.
 * X holds degrees 0..p-1; out gets degrees 0..p (out_0^0 = 0). Derivatives
 * of the family obey the same relations, so applying this twice gives the
 * second derivatives. */
static void ladder(int c, int p, const cplx* X, cplx* out) {
    out[0].re = 0.0; out[0].im = 0.0;
    for (int n = 1; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx lo = (m - 1 >= -(n - 1) && m - 1 <= n - 1) ? getc(X, n - 1, m - 1) : (cplx){0.0, 0.0};
            cplx hi = (m + 1 <= n - 1) ? getc(X, n - 1, m + 1) : (cplx){0.0, 0.0};
            cplx mid = (m <= n - 1) ? getc(X, n - 1, m) : (cplx){0.0, 0.0};
            cplx v;
            if (c == 0) {
                v.re = 0.5 * (lo.re - hi.re); v.im = 0.5 * (lo.im - hi.im);
            } else if (c == 1) {
                /* i (hi + lo) / 2 */
                v.re = -0.5 * (hi.im + lo.im); v.im = 0.5 * (hi.re + lo.re);
            } else {
                v = mid;
            }
            out[tri(n, m)] = v;
        }
}

/* Gradient of the regular harmonics: g[c][tri(n,m)] = d_c Upsilon_n^m(x,y,z),
 * n <= p. */
void orc_regular_grad(int p, double x, double y, double z, cplx* gx, cplx* gy, cplx* gz) {
    cplx R[ncoef(ORC_MAXP)];
    orc_regular(p > 0 ? p - 1 : 0, x, y, z, R);
    ladder(0, p, R, gx);
    ladder(1, p, R, gy);
    ladder(2, p, R, gz);
}

/* Multipoles of point dipoles (the far field of the jerk, see orc_jerk): a
 * dipole D at s has the potential D . grad_x (1 / |s - x|) =
 * -D . grad_s (1 / |x - s|), so with 1/|x - s| = sum conj(Upsilon(s - c))
 * Theta(x - c) its moments are M_n^m = -D . grad Upsilon_n^m(s - c). */
void orc_p2m_dipole(int p, int64_t n, const double* x, const double* y, const double* z,
                    const double* dx, const double* dy, const double* dz, double cx, double cy, double cz,
                    cplx* M) {
    cplx gx[ncoef(ORC_MAXP)], gy[ncoef(ORC_MAXP)], gz[ncoef(ORC_MAXP)];
    for (int64_t i = 0; i < n; ++i) {
        orc_regular_grad(p, x[i] - cx, y[i] - cy, z[i] - cz, gx, gy, gz);
        for (int k = 0; k < ncoef(p); ++k) {
            M[k].re -= dx[i] * gx[k].re + dy[i] * gy[k].re + dz[i] * gz[k].re;
            M[k].im -= dx[i] * gx[k].im + dy[i] * gy[k].im + dz[i] * gz[k].im;
        }
    }
}

/* Hessian of Psi(x) = sum_{n,m} conj(Upsilon_n^m(d)) F_n^m (= -phi without
 * G) at d: h = {xx, yy, zz, xy, xz, yz}, from the second derivatives of the
 * harmonics. */
void orc_l2p_hessian(int p, const cplx* F, double dx, double dy, double dz, double* h) {
    cplx g[3][ncoef(ORC_MAXP)], H[ncoef(ORC_MAXP)];
    orc_regular_grad(p > 0 ? p - 1 : 0, dx, dy, dz, g[0], g[1], g[2]);
    const int kc[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int e = 0; e < 6; ++e) {
        ladder(kc[e][1], p, g[kc[e][0]], H);
        double s = 0.0;
        for (int n = 0; n <= p; ++n)
            for (int m = -n; m <= n; ++m) s += cmul(cconj(getc(H, n, m)), getc(F, n, m)).re;
        h[e] = s;
    }
}

/* ------------------------------------------------------------ direct sum */

/* Plain O(N^2) FP64 sum over all j != i (the quantity the FMM approximates,
 * Sec. 2.3 and Sec. 3.1.1): a_i = G sum m_j (x_j - x_i)/|x_j - x_i|^3,
 * phi_i = -G sum m_j / |x_j - x_i|. Targets are the index list tgt. With
 * soft > 0 the kernel is Plummer-softened (Appendix B): |x_j - x_i|^2
 * becomes |x_j - x_i|^2 + soft^2 in both sums. */
void orc_direct(int64_t n, const double* x, const double* y, const double* z,
                const double* m, double G, double soft, int64_t ntgt, const int64_t* tgt,
                double* ax, double* ay, double* az, double* pot) {
    const double soft2 = soft * soft;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ntgt; ++t) {
        int64_t i = tgt ? tgt[t] : t;
        double sx = 0, sy = 0, sz = 0, sp = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (soft2 > 0.0) r2 = r2 + soft2;
            double r = sqrt(r2);
            double mr3 = m[j] / (r2 * r);
            sx += mr3 * dx; sy += mr3 * dy; sz += mr3 * dz;
            sp += m[j] / r;
        }
        ax[t] = G * sx; ay[t] = G * sy; az[t] = G * sz; pot[t] = -G * sp;
    }
}

/* Plain O(N^2) FP64 jerk, the time derivative of the direct-sum acceleration:
 * j_i = G sum_{j != i} m_j [v_ij / r^3 - 3 (r_ij . v_ij) r_ij / r^5],
 * r_ij = x_j - x_i, v_ij = v_j - v_i, r = |r_ij| (r^2 + soft^2 with
 * softening). */
void orc_direct_jerk(int64_t n, const double* x, const double* y, const double* z, const double* vx,
                     const double* vy, const double* vz, const double* m, double G, double soft,
                     int64_t ntgt, const int64_t* tgt, double* jx, double* jy, double* jz) {
    const double soft2 = soft * soft;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ntgt; ++t) {
        int64_t i = tgt ? tgt[t] : t;
        double sx = 0, sy = 0, sz = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double ux = vx[j] - vx[i], uy = vy[j] - vy[i], uz = vz[j] - vz[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (soft2 > 0.0) r2 = r2 + soft2;
            double r = sqrt(r2);
            double r3 = r2 * r, r5 = r3 * r2;
            double rv = dx * ux + dy * uy + dz * uz;
            sx += m[j] * (ux / r3 - 3.0 * rv * dx / r5);
            sy += m[j] * (uy / r3 - 3.0 * rv * dy / r5);
            sz += m[j] * (uz / r3 - 3.0 * rv * dz / r5);
        }
        jx[t] = G * sx; jy[t] = G * sy; jz[t] = G * sz;
    }
}

/* ----------------------------------------------- HOLD integrator (App. A) */

/* Step size of body i against body j (Appendix A): the smaller of the
 * free-fall time eta sqrt(r / a) with a = G (m_i + m_j) / r^2 and the fly-by
 * time eta r / v (r, v: separation and relative speed). With sym != 0 each is
 * replaced by tau / (1 - tau'/2) (Eq. step_symm), tau' its time derivative
 * along the two-body motion: for the free-fall time 1.5 tau (r . v) / r^2,
 * for the fly-by time tau ((r . v) / r^2 - (v . a_rel) / v^2) with the
 * two-body relative acceleration a_rel = -G (m_i + m_j) r / r^3. The
 * derivative is capped at 1 (the factor at 2) where the paper gives no rule.
 * Plain FP64, one IEEE operation per source operation (no contraction). */
double orc_tau_pair(double rx, double ry, double rz, double ux, double uy, double uz, double mij, double G,
                    double eta, int sym) {
    double r2 = rx * rx + ry * ry + rz * rz;
    double r = sqrt(r2);
    double v2 = ux * ux + uy * uy + uz * uz;
    double v = sqrt(v2);
    double gm = G * mij;
    double tff = eta * sqrt(r2 * r / gm);
    double tfl = v > 0.0 ? eta * r / v : INFINITY;
    if (sym) {
        double rv = rx * ux + ry * uy + rz * uz;
        double dff = 1.5 * tff * rv / r2;
        if (dff > 1.0) dff = 1.0;
        tff = tff / (1.0 - 0.5 * dff);
        if (v > 0.0) {
            double va = -gm * rv / (r2 * r);  /* v . a_rel */
            double dfl = tfl * (rv / r2 - va / v2);
            if (dfl > 1.0) dfl = 1.0;
            tfl = tfl / (1.0 - 0.5 * dfl);
        }
    }
    return tff < tfl ? tff : tfl;
}

/* tau_i = min over j in the set (j != i) of orc_tau_pair, for every member
 * i of the set idx[0..k). */
static void hold_taus(int64_t k, const int64_t* idx, const double* x, const double* y, const double* z,
                      const double* vx, const double* vy, const double* vz, const double* m, double G,
                      double eta, int sym, double* tau) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < k; ++a) {
        int64_t i = idx[a];
        double t = INFINITY;
        for (int64_t b = 0; b < k; ++b) {
            int64_t j = idx[b];
            if (j == i) continue;
            double tij = orc_tau_pair(x[j] - x[i], y[j] - y[i], z[j] - z[i], vx[j] - vx[i], vy[j] - vy[i],
                                      vz[j] - vz[i], m[i] + m[j], G, eta, sym);
            if (tij < t) t = tij;
        }
        tau[a] = t;
    }
}

/* tau_i over all n bodies (the set of every body). */
void orc_taus(int64_t n, const double* x, const double* y, const double* z, const double* vx, const double* vy,
              const double* vz, const double* m, double G, double eta, int sym, double* tau) {
    int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    hold_taus(n, all, x, y, z, vx, vy, vz, m, G, eta, sym, tau);
    free(all);
}

/* Acceleration of the sinks from the sources (index lists), direct FP64,
 * softened like orc_direct; a body does not act on itself. */
static void hold_accel(int64_t ns, const int64_t* sink, int64_t nsrc, const int64_t* src, const double* x,
                       const double* y, const double* z, const double* m, double G, double soft2, double* ax,
                       double* ay, double* az) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < ns; ++a) {
        int64_t i = sink[a];
        double sx = 0, sy = 0, sz = 0;
        for (int64_t b = 0; b < nsrc; ++b) {
            int64_t j = src[b];
            if (j == i) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (soft2 > 0.0) r2 = r2 + soft2;
            double r = sqrt(r2);
            double mr3 = m[j] / (r2 * r);
            sx += mr3 * dx; sy += mr3 * dy; sz += mr3 * dz;
        }
        ax[a] = G * sx; ay[a] = G * sy; az[a] = G * sz;
    }
}

typedef struct {
    double *x, *y, *z, *vx, *vy, *vz;
    const double* m;
    double G, soft2, eta, dt_min;
    int sym;
    int64_t n, kicks, force_evals, max_depth;
} hold_sys;

/* Kick of the slow system H_S = T_S + V_SS + V_FS over time h: slow bodies
 * feel all of P = S + F, fast bodies feel the slow ones only. */
static void hold_kick(hold_sys* s, int64_t ns, const int64_t* S, int64_t nf, const int64_t* F, const int64_t* P,
                      double h) {
    int64_t np = ns + nf;
    double* a = (double*)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    hold_accel(ns, S, np, P, s->x, s->y, s->z, s->m, s->G, s->soft2, a, a + ns, a + 2 * ns);
    for (int64_t q = 0; q < ns; ++q) {
        int64_t i = S[q];
        s->vx[i] += h * a[q]; s->vy[i] += h * a[ns + q]; s->vz[i] += h * a[2 * ns + q];
    }
    if (nf > 0) {
        hold_accel(nf, F, ns, S, s->x, s->y, s->z, s->m, s->G, s->soft2, a, a + nf, a + 2 * nf);
        for (int64_t q = 0; q < nf; ++q) {
            int64_t i = F[q];
            s->vx[i] += h * a[q]; s->vy[i] += h * a[nf + q]; s->vz[i] += h * a[2 * nf + q];
        }
    }
    s->kicks += 1;
    s->force_evals += ns * np + nf * ns;
    free(a);
}

/* Evolve the subsystem P = idx[0..k) under H_P = T_P + V_PP for time dt
 * (Appendix A, after Pelupessy et al. 2012): split P into fast bodies
 * (tau_i < dt, tau over pairs within P) and slow ones; evolve the fast
 * system for dt/2, kick-drift-kick the slow system (H_S, the slow bodies'
 * kinetic term, V_SS and V_FS), evolve the fast system for dt/2. Below
 * dt_min nothing is split further (a plain leapfrog step of P). */
static void hold_evolve(hold_sys* s, int64_t k, const int64_t* idx, double dt, int64_t depth) {
    if (k == 0) return;
    if (depth > s->max_depth) s->max_depth = depth;
    int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    int64_t* F = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    int64_t ns = 0, nf = 0;
    if (k > 1 && dt > s->dt_min) {
        double* tau = (double*)malloc(sizeof(double) * (size_t)k);
        hold_taus(k, idx, s->x, s->y, s->z, s->vx, s->vy, s->vz, s->m, s->G, s->eta, s->sym, tau);
        for (int64_t a = 0; a < k; ++a) {
            if (tau[a] < dt) F[nf++] = idx[a];
            else S[ns++] = idx[a];
        }
        free(tau);
    } else {
        for (int64_t a = 0; a < k; ++a) S[ns++] = idx[a];
    }
    for (int64_t a = 0; a < ns; ++a) P[a] = S[a];
    for (int64_t a = 0; a < nf; ++a) P[ns + a] = F[a];
    if (nf > 0) hold_evolve(s, nf, F, 0.5 * dt, depth + 1);
    if (ns > 0) {
        hold_kick(s, ns, S, nf, F, P, 0.5 * dt);
        for (int64_t a = 0; a < ns; ++a) {
            int64_t i = S[a];
            s->x[i] += dt * s->vx[i]; s->y[i] += dt * s->vy[i]; s->z[i] += dt * s->vz[i];
        }
        hold_kick(s, ns, S, nf, F, P, 0.5 * dt);
    }
    if (nf > 0) hold_evolve(s, nf, F, 0.5 * dt, depth + 1);
    free(S); free(F); free(P);
}

/* nsteps HOLD steps of size dt on all n bodies, in place. stats (may be
 * NULL): {slow-system kicks, pair force evaluations, deepest level}. */
void orc_hold(int64_t n, double* x, double* y, double* z, double* vx, double* vy, double* vz, const double* m,
              double G, double soft, double eta, int sym, double dt, int64_t nsteps, double dt_min,
              int64_t* stats) {
    hold_sys s = {x, y, z, vx, vy, vz, m, G, soft * soft, eta, dt_min, sym, n, 0, 0, 0};
    int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    for (int64_t t = 0; t < nsteps; ++t) hold_evolve(&s, n, all, dt, 0);
    free(all);
    if (stats) { stats[0] = s.kicks; stats[1] = s.force_evals; stats[2] = s.max_depth; }
}

/* Total energy sum m v^2 / 2 - G sum_{i<j} m_i m_j / |x_i - x_j| (softened
 * like orc_direct). */
double orc_energy(int64_t n, const double* x, const double* y, const double* z, const double* vx, const double* vy,
                  const double* vz, const double* m, double G, double soft) {
    double soft2 = soft * soft, ek = 0.0, ep = 0.0;
    for (int64_t i = 0; i < n; ++i) ek += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ep)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (soft2 > 0.0) r2 = r2 + soft2;
            s += m[j] / sqrt(r2);
        }
        ep += m[i] * s;
    }
    return ek - G * ep;
}

/* ------------------------------------------------------------- the solve */

typedef struct {
    /* inputs */
    int64_t n; int p; int leaf_size; double eps; double G;
    double soft2;  /* squared Plummer softening length (0: Newtonian) */
    int stage;   /* 1: tree; 2: + geometry, multipoles, f; 3: + lists; 4: full */
    int status;  /* 0 ok, -5 coincident particles */
    /* box and tree */
    double box[4];                      /* cube centre (3) and half-size */
    uint64_t* keys; int64_t* perm;      /* sorted keys, perm[sorted] = original */
    int32_t nnodes, nlevels;
    int32_t* level_start;               /* nlevels + 1 */
    int32_t *level, *begin, *end, *parent, *first_child, *nchild;
    /* sorted particles */
    double *xs, *ys, *zs, *ms;
    /* geometry */
    double *M, *S, *zc, *r;             /* S and zc: 3 per node */
    cplx* mult;                         /* ncoef(p) per node */
    double* P;                          /* p + 1 per node */
    float *f, *fmin;                    /* per sorted particle, per node */
    /* lists: pairs of node ids */
    int64_t nfar, nnear, nm2l, np2p, cap_far, cap_near, cap_m2l, cap_p2p;
    int32_t *far, *near, *m2l, *p2p;
    /* results */
    cplx* loc;                          /* ncoef(p) per node */
    double *ax, *ay, *az, *pot;         /* caller order */
    double mac_tests;
} orc_state;

/* -- tree ---------------------------------------------------------------- */

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* u = (const keyidx*)a;
    const keyidx* v = (const keyidx*)b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    return (u->idx < v->idx) ? -1 : (u->idx > v->idx);
}

static inline double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Bounding cube: centre c = (min+max)/2 per axis, half-size
 * h = max_axis (max-min)/2; quantise (x - (c-h)) / (2h) * 2^21, clamp to
 * [0, 2^21 - 1]; interleave with x in the high bit of each 3-bit digit. */
static void build_keys(orc_state* s, const double* x, const double* y, const double* z) {
    int64_t n = s->n;
    double mn[3] = {x[0], y[0], z[0]}, mx[3] = {x[0], y[0], z[0]};
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < mn[0]) mn[0] = x[i];
        if (x[i] > mx[0]) mx[0] = x[i];
        if (y[i] < mn[1]) mn[1] = y[i];
        if (y[i] > mx[1]) mx[1] = y[i];
        if (z[i] < mn[2]) mn[2] = z[i];
        if (z[i] > mx[2]) mx[2] = z[i];
    }
    double c[3], h = 0.0;
    for (int d = 0; d < 3; ++d) {
        c[d] = 0.5 * (mn[d] + mx[d]);
        double hd = 0.5 * (mx[d] - mn[d]);
        if (hd > h) h = hd;
    }
    if (h == 0.0) h = 1.0;
    s->box[0] = c[0]; s->box[1] = c[1]; s->box[2] = c[2]; s->box[3] = h;
    double lo[3] = {c[0] - h, c[1] - h, c[2] - h};
    double size = 2.0 * h;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double* pv[3] = {x, y, z};
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) {
            double t = (pv[d][i] - lo[d]) / size;
            double f = floor(t * 2097152.0);
            q[d] = (uint64_t)clampd(f, 0.0, 2097151.0);
        }
        uint64_t key = 0;
        for (int b = ORC_MAXLEVEL - 1; b >= 0; --b)
            key = (key << 3) | (((q[0] >> b) & 1) << 2) | (((q[1] >> b) & 1) << 1) | ((q[2] >> b) & 1);
        ki[i].key = key;
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < n; ++i) { s->keys[i] = ki[i].key; s->perm[i] = ki[i].idx; }
    free(ki);
}

static inline int digit_at(uint64_t key, int level) { /* level 1..21 */
    return (int)((key >> (3 * (ORC_MAXLEVEL - level))) & 7);
}

/* Octree: split a node while it holds more than leaf_size
 * particles and is above level 21; empty children are omitted; nodes are
 * numbered level by level and, within a level, in key order (breadth-first). */
static void build_nodes(orc_state* s) {
    int64_t n = s->n;
    int32_t cap = 1024;
    s->level = (int32_t*)malloc(sizeof(int32_t) * cap);
    s->begin = (int32_t*)malloc(sizeof(int32_t) * cap);
    s->end = (int32_t*)malloc(sizeof(int32_t) * cap);
    s->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    s->first_child = (int32_t*)malloc(sizeof(int32_t) * cap);
    s->nchild = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t nn = 1;
    s->level[0] = 0; s->begin[0] = 0; s->end[0] = (int32_t)n; s->parent[0] = -1;
    for (int32_t k = 0; k < nn; ++k) {
        s->first_child[k] = -1;
        s->nchild[k] = 0;
        int32_t b = s->begin[k], e = s->end[k], L = s->level[k];
        if (e - b <= s->leaf_size || L >= ORC_MAXLEVEL) continue;
        int32_t i = b;
        while (i < e) {
            int d = digit_at(s->keys[i], L + 1);
            int32_t j = i;
            while (j < e && digit_at(s->keys[j], L + 1) == d) ++j;
            if (nn == cap) {
                cap *= 2;
                s->level = (int32_t*)realloc(s->level, sizeof(int32_t) * cap);
                s->begin = (int32_t*)realloc(s->begin, sizeof(int32_t) * cap);
                s->end = (int32_t*)realloc(s->end, sizeof(int32_t) * cap);
                s->parent = (int32_t*)realloc(s->parent, sizeof(int32_t) * cap);
                s->first_child = (int32_t*)realloc(s->first_child, sizeof(int32_t) * cap);
                s->nchild = (int32_t*)realloc(s->nchild, sizeof(int32_t) * cap);
            }
            if (s->first_child[k] < 0) s->first_child[k] = nn;
            s->nchild[k] += 1;
            s->level[nn] = L + 1; s->begin[nn] = i; s->end[nn] = j; s->parent[nn] = k;
            ++nn;
            i = j;
        }
    }
    s->nnodes = nn;
    int32_t nl = s->level[nn - 1] + 1;
    s->nlevels = nl;
    s->level_start = (int32_t*)malloc(sizeof(int32_t) * (nl + 1));
    int32_t L = -1;
    for (int32_t k = 0; k < nn; ++k)
        while (L < s->level[k]) s->level_start[++L] = k;
    s->level_start[nl] = nn;
}

static inline int is_leaf(const orc_state* s, int32_t a) { return s->nchild[a] == 0; }

/* Coincident particles: two particles at exactly the same
 * position. They share a key, so they sit in the same run of equal keys. */
static int check_coincident(const orc_state* s) {
    int64_t n = s->n, i = 0;
    while (i < n) {
        int64_t j = i + 1;
        while (j < n && s->keys[j] == s->keys[i]) ++j;
        for (int64_t a = i; a < j; ++a)
            for (int64_t b = a + 1; b < j; ++b)
                if (s->xs[a] == s->xs[b] && s->ys[a] == s->ys[b] && s->zs[a] == s->zs[b]) return 1;
        i = j;
    }
    return 0;
}

/* Cell geometry: mass M_A, mass moment S_A = sum m x, the
 * expansion centre z_A = S_A / M_A (centre of mass) and size r_A. For a leaf
 * the sums run over its particles in sorted order and r_A is the largest
 * particle distance from z_A; an internal cell sums its children's M and S in
 * child order and takes r_A = max_C (|z_C - z_A| + r_C). */
static void cell_geometry(orc_state* s) {
    for (int32_t k = s->nnodes - 1; k >= 0; --k) {
        double M = 0, Sx = 0, Sy = 0, Sz = 0;
        if (is_leaf(s, k)) {
            for (int32_t i = s->begin[k]; i < s->end[k]; ++i) {
                M += s->ms[i];
                Sx += s->ms[i] * s->xs[i];
                Sy += s->ms[i] * s->ys[i];
                Sz += s->ms[i] * s->zs[i];
            }
        } else {
            for (int32_t c = s->first_child[k]; c < s->first_child[k] + s->nchild[k]; ++c) {
                M += s->M[c];
                Sx += s->S[3 * c]; Sy += s->S[3 * c + 1]; Sz += s->S[3 * c + 2];
            }
        }
        s->M[k] = M;
        s->S[3 * k] = Sx; s->S[3 * k + 1] = Sy; s->S[3 * k + 2] = Sz;
        double zx = Sx / M, zy = Sy / M, zz = Sz / M;
        s->zc[3 * k] = zx; s->zc[3 * k + 1] = zy; s->zc[3 * k + 2] = zz;
        double rr = 0.0;
        if (is_leaf(s, k)) {
            for (int32_t i = s->begin[k]; i < s->end[k]; ++i) {
                double dx = s->xs[i] - zx, dy = s->ys[i] - zy, dz = s->zs[i] - zz;
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (d > rr) rr = d;
            }
        } else {
            for (int32_t c = s->first_child[k]; c < s->first_child[k] + s->nchild[k]; ++c) {
                double dx = s->zc[3 * c] - zx, dy = s->zc[3 * c + 1] - zy, dz = s->zc[3 * c + 2] - zz;
                double d = sqrt(dx * dx + dy * dy + dz * dz) + s->r[c];
                if (d > rr) rr = d;
            }
        }
        s->r[k] = rr;
    }
}

/* Multipoles: P2M at leaves, M2M up in child order; then the degree norms
 * P_k^2 = sum_{m=-k}^{k} (k-m)!(k+m)! |M_k^m|^2 (Sec. 2.3). */
static void multipoles(orc_state* s) {
    int p = s->p, nc = ncoef(p);
    memset(s->mult, 0, sizeof(cplx) * (size_t)nc * s->nnodes);
    for (int32_t L = s->nlevels - 1; L >= 0; --L) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int32_t k = s->level_start[L]; k < s->level_start[L + 1]; ++k) {
            cplx* Mk = s->mult + (size_t)nc * k;
            const double* z = s->zc + 3 * k;
            if (is_leaf(s, k)) {
                int32_t b = s->begin[k];
                orc_p2m(p, s->end[k] - b, s->xs + b, s->ys + b, s->zs + b, s->ms + b, z[0], z[1], z[2], Mk);
            } else {
                for (int32_t c = s->first_child[k]; c < s->first_child[k] + s->nchild[k]; ++c) {
                    const double* zc = s->zc + 3 * c;
                    orc_m2m(p, s->mult + (size_t)nc * c, zc[0] - z[0], zc[1] - z[1], zc[2] - z[2], Mk);
                }
            }
        }
    }
    for (int32_t k = 0; k < s->nnodes; ++k) {
        const cplx* Mk = s->mult + (size_t)nc * k;
        for (int q = 0; q <= p; ++q) {
            cplx a = Mk[tri(q, 0)];
            double acc = FACT[q] * FACT[q] * (a.re * a.re + a.im * a.im);
            for (int m = 1; m <= q; ++m) {
                cplx b = Mk[tri(q, m)];
                acc += 2.0 * (FACT[q - m] * FACT[q + m]) * (b.re * b.re + b.im * b.im);
            }
            s->P[(size_t)(p + 1) * k + q] = sqrt(acc);
        }
    }
}

/* -- dual-tree walks ------------------------------------------------------- */

static void push_pair(int32_t** arr, int64_t* cnt, int64_t* cap, int32_t a, int32_t b) {
    if (*cnt == *cap) {
        *cap = (*cap == 0) ? 1024 : 2 * *cap;
        *arr = (int32_t*)realloc(*arr, sizeof(int32_t) * 2 * (size_t)*cap);
    }
    (*arr)[2 * *cnt] = a;
    (*arr)[2 * *cnt + 1] = b;
    ++*cnt;
}

/* Geometric part of the MAC: theta = (r_A + r_B)/r < 1 with
 * r = |z_A - z_B|, tested as r_A + r_B < r. */
static inline int theta_ok(const orc_state* s, int32_t a, int32_t b, double* r2out, double* rout) {
    const double* za = s->zc + 3 * a;
    const double* zb = s->zc + 3 * b;
    double dx = zb[0] - za[0], dy = zb[1] - za[1], dz = zb[2] - za[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    *r2out = r2; *rout = r;
    return s->r[a] + s->r[b] < r;
}

/* E_{A->B} M_A / r^2 of Sec. 2.3:
 *   [8 max(r_A,r_B)/(r_A+r_B)] * sum_{k=0}^{p} C(p,k) P_{k,A} r_B^{p-k} / (r^p r^2),
 * the sum in Horner form over k ascending, r^p by repeated multiplication,
 * and the prefactor taken as 4 when r_A + r_B = 0. */
static inline double mac_lhs(const orc_state* s, int32_t a, int32_t b, double r2, double r) {
    int p = s->p;
    double ra = s->r[a], rb = s->r[b];
    double sum = ra + rb;
    double pre = (sum > 0.0) ? 8.0 * (ra > rb ? ra : rb) / sum : 4.0;
    const double* Pa = s->P + (size_t)(p + 1) * a;
    double h = 0.0;
    for (int k = 0; k <= p; ++k) h = h * rb + BINOM[p][k] * Pa[k];
    double rp = 1.0;
    for (int k = 0; k < p; ++k) rp = rp * r;
    return pre * h / (rp * r2);
}

/* Bound on the softening the far field leaves out:
 * 1.5 M_A soft^2 / d_min^4, d_min = r - r_A - r_B (> 0 once theta < 1). */
static inline double soft_bound(const orc_state* s, int32_t a, int32_t b, double r) {
    double dmin = r - s->r[a] - s->r[b];
    double d2 = dmin * dmin;
    return 1.5 * s->M[a] * s->soft2 / (d2 * d2);
}

/* Full MAC of Sec. 2.3:
 * theta < 1 and E_{A->B} M_A/r^2 < eps f_B and E_{B->A} M_B/r^2 < eps f_A,
 * with f_A the minimum scalar force over the particles of A. With softening
 * each left side also carries soft_bound. */
static int mac_eps(orc_state* s, int32_t a, int32_t b) {
    double r2, r;
    s->mac_tests += 1.0;
    if (!theta_ok(s, a, b, &r2, &r)) return 0;
    double lab = mac_lhs(s, a, b, r2, r);
    double lba = mac_lhs(s, b, a, r2, r);
    if (s->soft2 > 0.0) {
        lab = lab + soft_bound(s, a, b, r);
        lba = lba + soft_bound(s, b, a, r);
    }
    return lab < s->eps * (double)s->fmin[b] && lba < s->eps * (double)s->fmin[a];
}

/* Dual-tree walk: a self pair of a leaf goes to P2P, of an
 * internal cell to the pairs (C_i, C_j), i <= j, of its children; another
 * pair is accepted by the MAC, or, if both cells are leaves, goes to P2P, or
 * else the cell with the larger r is split (A on a tie; never a leaf). */
static void walk(orc_state* s, int32_t a, int32_t b, int mode) {
    if (a == b) {
        if (is_leaf(s, a)) {
            if (mode == 0) push_pair(&s->near, &s->nnear, &s->cap_near, a, a);
            else push_pair(&s->p2p, &s->np2p, &s->cap_p2p, a, a);
            return;
        }
        int32_t c0 = s->first_child[a], nc = s->nchild[a];
        for (int32_t i = c0; i < c0 + nc; ++i)
            for (int32_t j = i; j < c0 + nc; ++j) walk(s, i, j, mode);
        return;
    }
    int acc;
    if (mode == 0) {
        double r2, r;
        acc = theta_ok(s, a, b, &r2, &r);
    } else {
        acc = mac_eps(s, a, b);
    }
    if (acc) {
        if (mode == 0) push_pair(&s->far, &s->nfar, &s->cap_far, a, b);
        else push_pair(&s->m2l, &s->nm2l, &s->cap_m2l, a, b);
        return;
    }
    int la = is_leaf(s, a), lb = is_leaf(s, b);
    if (la && lb) {
        if (mode == 0) push_pair(&s->near, &s->nnear, &s->cap_near, a, b);
        else push_pair(&s->p2p, &s->np2p, &s->cap_p2p, a, b);
        return;
    }
    int split_a = lb ? 1 : (la ? 0 : (s->r[a] >= s->r[b]));
    if (split_a) {
        for (int32_t c = s->first_child[a]; c < s->first_child[a] + s->nchild[a]; ++c) walk(s, c, b, mode);
    } else {
        for (int32_t c = s->first_child[b]; c < s->first_child[b] + s->nchild[b]; ++c) walk(s, a, c, mode);
    }
}

/* Per-target partner lists, partners sorted ascending (CSR). Each unordered
 * pair (a, b) lists b as a partner of a and a of b; a self pair lists a once. */
static void partner_csr(int32_t nnodes, int64_t npairs, const int32_t* pairs,
                        int64_t** off_out, int32_t** idx_out) {
    int64_t* off = (int64_t*)calloc((size_t)nnodes + 1, sizeof(int64_t));
    for (int64_t q = 0; q < npairs; ++q) {
        int32_t a = pairs[2 * q], b = pairs[2 * q + 1];
        off[a + 1]++;
        if (a != b) off[b + 1]++;
    }
    for (int32_t k = 0; k < nnodes; ++k) off[k + 1] += off[k];
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[nnodes] > 0 ? off[nnodes] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnodes);
    memcpy(fill, off, sizeof(int64_t) * (size_t)nnodes);
    for (int64_t q = 0; q < npairs; ++q) {
        int32_t a = pairs[2 * q], b = pairs[2 * q + 1];
        idx[fill[a]++] = b;
        if (a != b) idx[fill[b]++] = a;
    }
    free(fill);
    for (int32_t k = 0; k < nnodes; ++k) {
        /* insertion sort: lists are short */
        for (int64_t i = off[k] + 1; i < off[k + 1]; ++i) {
            int32_t v = idx[i];
            int64_t j = i - 1;
            while (j >= off[k] && idx[j] > v) { idx[j + 1] = idx[j]; --j; }
            idx[j + 1] = v;
        }
    }
    *off_out = off;
    *idx_out = idx;
}

/* Scalar-force estimate f_i = sum_{j != i} m_j / |x_i - x_j|^2 (Sec. 2.3),
 * in FP32 with a fixed order (the paper fixes neither):
 *  - a walk with theta < 1 only; an accepted pair adds M_A/r^2 to cell B and
 *    M_B/r^2 to cell A, with r^2 from the FP32-rounded centre offsets;
 *    a cell sums its terms over its partners in ascending node order;
 *  - these far terms are pushed down: g(child) = g(parent) + far(child);
 *  - near leaf pairs are summed particle by particle over partner leaves in
 *    ascending order and their particles in sorted order, skipping j = i,
 *    on FP32 coordinates relative to the cube centre; with softening the
 *    term is the softened force magnitude m r / (r^2 + soft^2)^(3/2);
 *  - f_i = g(leaf) + near_i, and fmin(A) = min over the particles of A.
 * G cancels from both sides of the MAC and is left out. */
static void scalar_force(orc_state* s) {
    int32_t nn = s->nnodes;
    float* far = (float*)calloc((size_t)nn, sizeof(float));
    float* g = (float*)calloc((size_t)nn, sizeof(float));
    int64_t* off; int32_t* idx;
    partner_csr(nn, s->nfar, s->far, &off, &idx);
    for (int32_t b = 0; b < nn; ++b) {
        float acc = 0.0f;
        const double* zb = s->zc + 3 * b;
        for (int64_t q = off[b]; q < off[b + 1]; ++q) {
            int32_t a = idx[q];
            const double* za = s->zc + 3 * a;
            float dx = (float)(za[0] - zb[0]), dy = (float)(za[1] - zb[1]), dz = (float)(za[2] - zb[2]);
            float r2 = dx * dx + dy * dy + dz * dz;
            acc = acc + (float)s->M[a] / r2;
        }
        far[b] = acc;
    }
    free(off); free(idx);
    for (int32_t k = 0; k < nn; ++k) g[k] = (k == 0) ? far[0] : g[s->parent[k]] + far[k];

    int64_t n = s->n;
    float* xf = (float*)malloc(sizeof(float) * 4 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        xf[4 * i] = (float)(s->xs[i] - s->box[0]);
        xf[4 * i + 1] = (float)(s->ys[i] - s->box[1]);
        xf[4 * i + 2] = (float)(s->zs[i] - s->box[2]);
        xf[4 * i + 3] = (float)s->ms[i];
    }
    partner_csr(nn, s->nnear, s->near, &off, &idx);
    const float soft2f = (float)s->soft2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t b = 0; b < nn; ++b) {
        if (!is_leaf(s, b)) continue;
        for (int32_t i = s->begin[b]; i < s->end[b]; ++i) {
            float acc = 0.0f;
            float xi = xf[4 * i], yi = xf[4 * i + 1], zi = xf[4 * i + 2];
            for (int64_t q = off[b]; q < off[b + 1]; ++q) {
                int32_t a = idx[q];
                for (int32_t j = s->begin[a]; j < s->end[a]; ++j) {
                    if (j == i) continue;
                    float dx = xf[4 * j] - xi, dy = xf[4 * j + 1] - yi, dz = xf[4 * j + 2] - zi;
                    float r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 > 0.0f)) continue;
                    if (soft2f > 0.0f) {
                        float s2 = r2 + soft2f;
                        acc = acc + xf[4 * j + 3] * sqrtf(r2) / (s2 * sqrtf(s2));
                    } else {
                        acc = acc + xf[4 * j + 3] / r2;
                    }
                }
            }
            s->f[i] = g[b] + acc;
        }
    }
    free(off); free(idx); free(xf);
    for (int32_t k = nn - 1; k >= 0; --k) {
        float mn;
        if (is_leaf(s, k)) {
            mn = s->f[s->begin[k]];
            for (int32_t i = s->begin[k] + 1; i < s->end[k]; ++i)
                if (s->f[i] < mn) mn = s->f[i];
        } else {
            int32_t c0 = s->first_child[k];
            mn = s->fmin[c0];
            for (int32_t c = c0 + 1; c < c0 + s->nchild[k]; ++c)
                if (s->fmin[c] < mn) mn = s->fmin[c];
        }
        s->fmin[k] = mn;
    }
    free(far); free(g);
}

/* Far field: M2L both ways for every accepted pair, gathered
 * per target; L2L down; L2P per particle. Near field: P2P over leaf pairs,
 * both directions, and within a leaf over j != i, softened when soft > 0. */
static void forces(orc_state* s) {
    int p = s->p, nc = ncoef(p);
    int32_t nn = s->nnodes;
    int64_t n = s->n;
    memset(s->loc, 0, sizeof(cplx) * (size_t)nc * nn);
    int64_t* off; int32_t* idx;
    partner_csr(nn, s->nm2l, s->m2l, &off, &idx);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t b = 0; b < nn; ++b) {
        const double* zb = s->zc + 3 * b;
        for (int64_t q = off[b]; q < off[b + 1]; ++q) {
            int32_t a = idx[q];
            const double* za = s->zc + 3 * a;
            orc_m2l(p, s->mult + (size_t)nc * a, za[0] - zb[0], za[1] - zb[1], za[2] - zb[2],
                    s->loc + (size_t)nc * b);
        }
    }
    free(off); free(idx);
    for (int32_t L = 1; L < s->nlevels; ++L) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int32_t k = s->level_start[L]; k < s->level_start[L + 1]; ++k) {
            int32_t par = s->parent[k];
            const double* zk = s->zc + 3 * k;
            const double* zp = s->zc + 3 * par;
            orc_l2l(p, s->loc + (size_t)nc * par, zk[0] - zp[0], zk[1] - zp[1], zk[2] - zp[2],
                    s->loc + (size_t)nc * k);
        }
    }
    double* fx = (double*)calloc((size_t)n, sizeof(double));
    double* fy = (double*)calloc((size_t)n, sizeof(double));
    double* fz = (double*)calloc((size_t)n, sizeof(double));
    double* fp = (double*)calloc((size_t)n, sizeof(double));
    partner_csr(nn, s->np2p, s->p2p, &off, &idx);
#pragma omp parallel for schedule(dynamic, 8)
    for (int32_t b = 0; b < nn; ++b) {
        if (!is_leaf(s, b)) continue;
        const double* zb = s->zc + 3 * b;
        for (int32_t i = s->begin[b]; i < s->end[b]; ++i) {
            double phi, ax, ay, az;
            orc_l2p(p, s->loc + (size_t)nc * b, s->xs[i] - zb[0], s->ys[i] - zb[1], s->zs[i] - zb[2],
                    &phi, &ax, &ay, &az);
            double sx = 0, sy = 0, sz = 0, sp = 0;
            for (int64_t q = off[b]; q < off[b + 1]; ++q) {
                int32_t a = idx[q];
                for (int32_t j = s->begin[a]; j < s->end[a]; ++j) {
                    if (j == i) continue;
                    double dx = s->xs[j] - s->xs[i], dy = s->ys[j] - s->ys[i], dz = s->zs[j] - s->zs[i];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (s->soft2 > 0.0) r2 = r2 + s->soft2;
                    double r = sqrt(r2);
                    double mr3 = s->ms[j] / (r2 * r);
                    sx += mr3 * dx; sy += mr3 * dy; sz += mr3 * dz;
                    sp += s->ms[j] / r;
                }
            }
            fx[i] = ax + sx; fy[i] = ay + sy; fz[i] = az + sz; fp[i] = phi - sp;
        }
    }
    free(off); free(idx);
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = s->perm[i];
        s->ax[o] = s->G * fx[i];
        s->ay[o] = s->G * fy[i];
        s->az[o] = s->G * fz[i];
        s->pot[o] = s->G * fp[i];
    }
    free(fx); free(fy); free(fz); free(fp);
}

/* Jerk (the time derivative of the acceleration) on the tree and lists of a
 * full solve. With T(y) = grad_y (y / |y|^3) = -grad grad (1 / |y|), the jerk
 * G sum_j m_j T(x_j - x_i) (v_j - v_i) splits into three parts:
 *   j_i = G [ -grad chi(x_i) + H(x_i) v_i + near_i ]
 *  - chi(x) = sum_j m_j v_j . grad_x (1 / |x_j - x|) is the potential of
 *    point dipoles m_j v_j; its far part is one more expansion through the
 *    same tree and lists (dipole P2M, M2M, M2L both ways, L2L) and its
 *    gradient comes from the degree-1 local coefficients, as the
 *    acceleration does;
 *  - H = grad grad Psi is the Hessian of Psi = sum_j m_j / |x_j - x| from the
 *    solve's own local expansion (orc_l2p_hessian);
 *  - near_i is the direct jerk over the P2P leaf pairs (softened as P2P is).
 * Velocities and the outputs are in the caller's order. */
int orc_jerk(orc_state* s, const double* vx, const double* vy, const double* vz,
             double* jx_out, double* jy_out, double* jz_out) {
    if (s->status != 0 || s->stage < 4) return -1;
    int p = s->p, nc = ncoef(p);
    int32_t nn = s->nnodes;
    int64_t n = s->n;
    double* vs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* ds = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = s->perm[i];
        vs[i] = vx[o]; vs[n + i] = vy[o]; vs[2 * n + i] = vz[o];
        ds[i] = s->ms[i] * vx[o]; ds[n + i] = s->ms[i] * vy[o]; ds[2 * n + i] = s->ms[i] * vz[o];
    }
    cplx* mj = (cplx*)calloc((size_t)nc * nn, sizeof(cplx));
    cplx* lj = (cplx*)calloc((size_t)nc * nn, sizeof(cplx));
    for (int32_t L = s->nlevels - 1; L >= 0; --L) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int32_t k = s->level_start[L]; k < s->level_start[L + 1]; ++k) {
            cplx* Mk = mj + (size_t)nc * k;
            const double* z = s->zc + 3 * k;
            if (is_leaf(s, k)) {
                int32_t b = s->begin[k];
                orc_p2m_dipole(p, s->end[k] - b, s->xs + b, s->ys + b, s->zs + b, ds + b, ds + n + b,
                               ds + 2 * n + b, z[0], z[1], z[2], Mk);
            } else {
                for (int32_t c = s->first_child[k]; c < s->first_child[k] + s->nchild[k]; ++c) {
                    const double* zc = s->zc + 3 * c;
                    orc_m2m(p, mj + (size_t)nc * c, zc[0] - z[0], zc[1] - z[1], zc[2] - z[2], Mk);
                }
            }
        }
    }
    int64_t* off; int32_t* idx;
    partner_csr(nn, s->nm2l, s->m2l, &off, &idx);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t b = 0; b < nn; ++b) {
        const double* zb = s->zc + 3 * b;
        for (int64_t q = off[b]; q < off[b + 1]; ++q) {
            int32_t a = idx[q];
            const double* za = s->zc + 3 * a;
            orc_m2l(p, mj + (size_t)nc * a, za[0] - zb[0], za[1] - zb[1], za[2] - zb[2], lj + (size_t)nc * b);
        }
    }
    free(off); free(idx);
    for (int32_t L = 1; L < s->nlevels; ++L) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int32_t k = s->level_start[L]; k < s->level_start[L + 1]; ++k) {
            int32_t par = s->parent[k];
            const double* zk = s->zc + 3 * k;
            const double* zp = s->zc + 3 * par;
            orc_l2l(p, lj + (size_t)nc * par, zk[0] - zp[0], zk[1] - zp[1], zk[2] - zp[2], lj + (size_t)nc * k);
        }
    }
    partner_csr(nn, s->np2p, s->p2p, &off, &idx);
#pragma omp parallel for schedule(dynamic, 8)
    for (int32_t b = 0; b < nn; ++b) {
        if (!is_leaf(s, b)) continue;
        const double* zb = s->zc + 3 * b;
        for (int32_t i = s->begin[b]; i < s->end[b]; ++i) {
            double dx = s->xs[i] - zb[0], dy = s->ys[i] - zb[1], dz = s->zs[i] - zb[2];
            double phi, gx, gy, gz, h[6];
            orc_l2p(p, lj + (size_t)nc * b, dx, dy, dz, &phi, &gx, &gy, &gz);
            orc_l2p_hessian(p, s->loc + (size_t)nc * b, dx, dy, dz, h);
            double vix = vs[i], viy = vs[n + i], viz = vs[2 * n + i];
            double fx = -gx + h[0] * vix + h[3] * viy + h[4] * viz;
            double fy = -gy + h[3] * vix + h[1] * viy + h[5] * viz;
            double fz = -gz + h[4] * vix + h[5] * viy + h[2] * viz;
            double sx = 0, sy = 0, sz = 0;
            for (int64_t q = off[b]; q < off[b + 1]; ++q) {
                int32_t a = idx[q];
                for (int32_t j = s->begin[a]; j < s->end[a]; ++j) {
                    if (j == i) continue;
                    double rx = s->xs[j] - s->xs[i], ry = s->ys[j] - s->ys[i], rz = s->zs[j] - s->zs[i];
                    double ux = vs[j] - vix, uy = vs[n + j] - viy, uz = vs[2 * n + j] - viz;
                    double r2 = rx * rx + ry * ry + rz * rz;
                    if (s->soft2 > 0.0) r2 = r2 + s->soft2;
                    double r = sqrt(r2);
                    double r3 = r2 * r, r5 = r3 * r2;
                    double rv = rx * ux + ry * uy + rz * uz;
                    sx += s->ms[j] * (ux / r3 - 3.0 * rv * rx / r5);
                    sy += s->ms[j] * (uy / r3 - 3.0 * rv * ry / r5);
                    sz += s->ms[j] * (uz / r3 - 3.0 * rv * rz / r5);
                }
            }
            int64_t o = s->perm[i];
            jx_out[o] = s->G * (fx + sx);
            jy_out[o] = s->G * (fy + sy);
            jz_out[o] = s->G * (fz + sz);
        }
    }
    free(off); free(idx);
    free(mj); free(lj); free(vs); free(ds);
    return 0;
}

void orc_free(orc_state* s);

/* Run the solve up to `stage` and keep every intermediate for inspection. */
orc_state* orc_run(int64_t n, const double* x, const double* y, const double* z, const double* m,
                   int p, double eps, int leaf_size, double G, double soft, int stage) {
    init_tables();
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    s->n = n; s->p = p; s->leaf_size = leaf_size; s->eps = eps; s->G = G; s->stage = stage;
    s->soft2 = soft * soft;
    if (n < 1 || p < 1 || p > ORC_MAXP || leaf_size < 1) { s->status = -1; return s; }
    s->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    s->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    build_keys(s, x, y, z);
    s->xs = (double*)malloc(sizeof(double) * (size_t)n);
    s->ys = (double*)malloc(sizeof(double) * (size_t)n);
    s->zs = (double*)malloc(sizeof(double) * (size_t)n);
    s->ms = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        s->xs[i] = x[s->perm[i]]; s->ys[i] = y[s->perm[i]];
        s->zs[i] = z[s->perm[i]]; s->ms[i] = m[s->perm[i]];
    }
    build_nodes(s);
    if (check_coincident(s)) { s->status = -5; return s; }
    if (stage < 2) return s;
    int32_t nn = s->nnodes;
    s->M = (double*)malloc(sizeof(double) * nn);
    s->S = (double*)malloc(sizeof(double) * 3 * nn);
    s->zc = (double*)malloc(sizeof(double) * 3 * nn);
    s->r = (double*)malloc(sizeof(double) * nn);
    s->mult = (cplx*)malloc(sizeof(cplx) * (size_t)ncoef(p) * nn);
    s->P = (double*)malloc(sizeof(double) * (size_t)(p + 1) * nn);
    s->f = (float*)malloc(sizeof(float) * (size_t)n);
    s->fmin = (float*)malloc(sizeof(float) * nn);
    cell_geometry(s);
    multipoles(s);
    walk(s, 0, 0, 0);
    scalar_force(s);
    if (stage < 3) return s;
    walk(s, 0, 0, 1);
    if (stage < 4) return s;
    s->loc = (cplx*)malloc(sizeof(cplx) * (size_t)ncoef(p) * nn);
    s->ax = (double*)malloc(sizeof(double) * (size_t)n);
    s->ay = (double*)malloc(sizeof(double) * (size_t)n);
    s->az = (double*)malloc(sizeof(double) * (size_t)n);
    s->pot = (double*)malloc(sizeof(double) * (size_t)n);
    forces(s);
    return s;
}

void orc_free(orc_state* s) {
    if (!s) return;
    void* ptrs[] = {s->keys, s->perm, s->level_start, s->level, s->begin, s->end, s->parent,
                    s->first_child, s->nchild, s->xs, s->ys, s->zs, s->ms, s->M, s->S, s->zc, s->r,
                    s->mult, s->P, s->f, s->fmin, s->far, s->near, s->m2l, s->p2p, s->loc,
                    s->ax, s->ay, s->az, s->pot};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(s);
}

/* -- accessors for the ctypes shim ---------------------------------------- */

int orc_status(const orc_state* s) { return s->status; }
int32_t orc_nnodes(const orc_state* s) { return s->nnodes; }
int32_t orc_nlevels(const orc_state* s) { return s->nlevels; }
double orc_mac_tests(const orc_state* s) { return s->mac_tests; }
int64_t orc_npairs(const orc_state* s, int which) {
    switch (which) {
        case 0: return s->nfar;
        case 1: return s->nnear;
        case 2: return s->nm2l;
        default: return s->np2p;
    }
}

#define COPY(dst, src, bytes) do { if (src) memcpy(dst, src, bytes); } while (0)

/* Copy an intermediate out. which: 0 keys, 1 perm, 2 level, 3 begin, 4 end,
 * 5 parent, 6 first_child, 7 nchild, 8 M, 9 zc(3/node), 10 r, 11 P((p+1)/node),
 * 12 f, 13 fmin, 14 far, 15 near, 16 m2l, 17 p2p, 18 multipoles (re,im),
 * 19 locals (re,im), 20 ax, 21 ay, 22 az, 23 pot, 24 box(4), 25 level_start,
 * 26 S(3/node). */
int orc_copy(const orc_state* s, int which, void* dst) {
    size_t n = (size_t)s->n, nn = (size_t)s->nnodes, nc = (size_t)ncoef(s->p);
    switch (which) {
        case 0: COPY(dst, s->keys, 8 * n); break;
        case 1: COPY(dst, s->perm, 8 * n); break;
        case 2: COPY(dst, s->level, 4 * nn); break;
        case 3: COPY(dst, s->begin, 4 * nn); break;
        case 4: COPY(dst, s->end, 4 * nn); break;
        case 5: COPY(dst, s->parent, 4 * nn); break;
        case 6: COPY(dst, s->first_child, 4 * nn); break;
        case 7: COPY(dst, s->nchild, 4 * nn); break;
        case 8: COPY(dst, s->M, 8 * nn); break;
        case 9: COPY(dst, s->zc, 24 * nn); break;
        case 10: COPY(dst, s->r, 8 * nn); break;
        case 11: COPY(dst, s->P, 8 * nn * (size_t)(s->p + 1)); break;
        case 12: COPY(dst, s->f, 4 * n); break;
        case 13: COPY(dst, s->fmin, 4 * nn); break;
        case 14: COPY(dst, s->far, 8 * (size_t)s->nfar); break;
        case 15: COPY(dst, s->near, 8 * (size_t)s->nnear); break;
        case 16: COPY(dst, s->m2l, 8 * (size_t)s->nm2l); break;
        case 17: COPY(dst, s->p2p, 8 * (size_t)s->np2p); break;
        case 18: COPY(dst, s->mult, 16 * nn * nc); break;
        case 19: COPY(dst, s->loc, 16 * nn * nc); break;
        case 20: COPY(dst, s->ax, 8 * n); break;
        case 21: COPY(dst, s->ay, 8 * n); break;
        case 22: COPY(dst, s->az, 8 * n); break;
        case 23: COPY(dst, s->pot, 8 * n); break;
        case 24: memcpy(dst, s->box, 32); break;
        case 25: COPY(dst, s->level_start, 4 * (size_t)(s->nlevels + 1)); break;
        case 26: COPY(dst, s->S, 24 * nn); break;
        default: return -1;
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the oracle's parallel loops (for timing it on one core). */
void orc_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* The two sides of the MAC for a pair of cells: out = {E_{A->B} M_A/r^2,
 * E_{B->A} M_B/r^2, eps f_B, eps f_A, theta-test passed, softening bound
 * A->B, softening bound B->A} (the bounds are 0 without softening or when
 * the theta test fails). */
void orc_mac_values(orc_state* s, int32_t a, int32_t b, double* out) {
    double r2, r;
    int ok = theta_ok(s, a, b, &r2, &r);
    out[0] = mac_lhs(s, a, b, r2, r);
    out[1] = mac_lhs(s, b, a, r2, r);
    out[2] = s->eps * (double)s->fmin[b];
    out[3] = s->eps * (double)s->fmin[a];
    out[4] = (double)ok;
    out[5] = (ok && s->soft2 > 0.0) ? soft_bound(s, a, b, r) : 0.0;
    out[6] = (ok && s->soft2 > 0.0) ? soft_bound(s, b, a, r) : 0.0;
}
