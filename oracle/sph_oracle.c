/*
 * sph_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64, brute-force O(N^2) CPU restatement of the SPH sums of
 * Theuns, Chalk, Schaller & Gonnet 2015 ("Swift: task-based hydrodynamics and
 * gravity for cosmological simulations"), Sec. 2, and of the near-field part of
 * its gravity (Sec. 3.2, Eq. 3; see orc_grav_p2p).  Only tests/, the smoke check
 * of __graft_entry__ and the CPU-baseline leg of bench.py may load this file.
 * The CUDA library never includes, links or calls it, and it shares no code
 * with the CUDA library.
 *
 * Every sum runs over ALL particles j in index order, with the periodic
 * minimal-image separation; there are no cells, no sorting, no pruning.  A
 * candidate list (all j within an upper radius, in index order) is cached
 * inside the smoothing-length solve only: the terms it drops are exactly zero
 * (W and dW/dq vanish for q >= 1), so the sums are unchanged bit for bit.
 *
 * Readings of the paper (the paper gives Eq. 1 only in illustrative form and
 * defers the force law to the Gadget-2 formulation it cites):
 *   - h is the kernel SUPPORT radius: W(q) = 0 for q > 1 (Sec. 2, below Eq. 2).
 *   - W(r,h) = h^-3 w(r/h), w = (8/pi){1-6q^2+6q^3 (q<=1/2); 2(1-q)^3 (1/2<q<=1)},
 *     the cubic spline of Monaghan & Lattanzio 1985 (not in the paper).
 *   - Eq. 1 density includes the self term j = i.
 *   - h is set by a weighted neighbour count (Sec. 2, after Eq. 2):
 *     N_w(h) = (4 pi / 3) sum_j w(r_ij / h) = N_ngb.
 *   - The equation of state (Sec. 2 gives pressure as a function of density and
 *     temperature without naming one): ideal gas,
 *     P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u).
 *   - The force law the paper defers to Gadget-2 (Sec. 2, after Eq. 2): the
 *     grad-h conservative equations of motion of Springel & Hernquist 2002 /
 *     Springel 2005, with the signal-velocity artificial viscosity
 *     (Monaghan 1997) and the Balsara 1995 switch.
 * Compile with -ffp-contract=off so x86 and Arm give the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_SIGMA (8.0 / ORC_PI) /* 3-D cubic-spline normalisation */
#define ORC_FOUR_PI_3 (4.0 * ORC_PI / 3.0)

/* ---- kernel shape (Sec. 2: a bell-shaped kernel that vanishes beyond h) ---- */

double orc_w(double q)
{
    if (q < 0.0) q = -q;
    if (q <= 0.5) return ORC_SIGMA * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    if (q <= 1.0) {
        double t = 1.0 - q;
        return ORC_SIGMA * 2.0 * t * t * t;
    }
    return 0.0;
}

/* dw/dq */
double orc_dw(double q)
{
    if (q < 0.0) q = -q;
    if (q <= 0.5) return ORC_SIGMA * (-12.0 * q + 18.0 * q * q);
    if (q <= 1.0) {
        double t = 1.0 - q;
        return ORC_SIGMA * (-6.0) * t * t;
    }
    return 0.0;
}

/* ---- periodic box (Sec. 2: the volume repeats periodically in every axis) ---- */

/* Wrap into [0, box): positions already inside are returned unchanged; others are
 * shifted by box*floor(x/box), then corrected by one box if rounding left them
 * just outside (and set to 0 if still outside). */
double orc_wrap1(double v, double box)
{
    if (v >= 0.0 && v < box) return v;
    double w = v - box * floor(v / box);
    if (w < 0.0) w += box;
    if (w >= box) w -= box;
    if (w < 0.0 || w >= box) w = 0.0;
    return w;
}

void orc_wrap(int64_t n, double box, double *x)
{
    for (int64_t i = 0; i < n; ++i) x[i] = orc_wrap1(x[i], box);
}

static inline double min_image(double d, double box)
{
    return d - box * rint(d / box);
}

/* Cell of a (wrapped) position on an nc^3 grid: floor(x * (nc/box)) per axis,
 * clamped to nc-1; key = (iz*nc + iy)*nc + ix.  Sec. 3.1: cubic cells. */
int64_t orc_cell_key(double x, double y, double z, double box, int64_t nc)
{
    double s = (double)nc / box;
    int64_t ix = (int64_t)floor(x * s), iy = (int64_t)floor(y * s), iz = (int64_t)floor(z * s);
    if (ix < 0) ix = 0;
    if (iy < 0) iy = 0;
    if (iz < 0) iz = 0;
    if (ix > nc - 1) ix = nc - 1;
    if (iy > nc - 1) iy = nc - 1;
    if (iz > nc - 1) iz = nc - 1;
    return (iz * nc + iy) * nc + ix;
}

/* splitmix64 finaliser: order-independent fingerprint of a neighbour set. */
static inline uint64_t orc_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_hash_id(uint64_t id) { return orc_mix64(id); }

typedef struct {
    int64_t n;
    double box;
    const double *x, *y, *z, *vx, *vy, *vz, *m;
} orc_parts;

static inline double sep2(const orc_parts *p, int64_t i, int64_t j, double *dx, double *dy, double *dz)
{
    double ax = min_image(p->x[i] - p->x[j], p->box);
    double ay = min_image(p->y[i] - p->y[j], p->box);
    double az = min_image(p->z[i] - p->z[j], p->box);
    *dx = ax;
    *dy = ay;
    *dz = az;
    return ax * ax + ay * ay + az * az;
}

/*
 * Eq. 1 and its companions at a GIVEN smoothing length h_i, for one target i:
 *   rho_i       = sum_j m_j h^-3 w(q)                       (Eq. 1, self term included)
 *   nw_i        = (4pi/3) sum_j w(q)                        (weighted neighbour number)
 *   dnw_dh_i    = (4pi/3) sum_j -q w'(q) / h
 *   drho_dh_i   = sum_j m_j h^-4 (-3 w(q) - q w'(q))
 *   divv_i      = -(1/rho_i) sum_j m_j v_ij . grad_i W_ij
 *   curl_i      =  (1/rho_i) sum_j m_j v_ij x grad_i W_ij
 *   n_ngb_i     = #{ j != i : r_ij < h_i }
 * with grad_i W_ij = (r_i - r_j)/r * h^-4 w'(q), q = r/h, r the minimal-image distance.
 */
static void density_one(const orc_parts *p, int64_t i, double h, const int64_t *cand, int64_t ncand,
                        const uint64_t *ids, double out[9], int64_t *nngb, uint64_t *hash)
{
    double h2 = h * h, hinv = 1.0 / h;
    double hinv3 = hinv * hinv * hinv, hinv4 = hinv3 * hinv;
    double rho = 0, sw = 0, sqdw = 0, drho = 0, dv = 0, cx = 0, cy = 0, cz = 0;
    int64_t cnt = 0;
    uint64_t hh = 0;
    int64_t nj = cand ? ncand : p->n;
    for (int64_t k = 0; k < nj; ++k) {
        int64_t j = cand ? cand[k] : k;
        double dx, dy, dz;
        double r2 = sep2(p, i, j, &dx, &dy, &dz);
        if (j != i && !(r2 < h2)) continue;
        double r = sqrt(r2);
        double q = r * hinv;
        double w = orc_w(q), dw = orc_dw(q);
        double mj = p->m[j];
        rho += mj * hinv3 * w;
        sw += w;
        sqdw += -q * dw;
        drho += mj * hinv4 * (-3.0 * w - q * dw);
        if (j != i) {
            ++cnt;
            hh += orc_mix64(ids ? ids[j] : (uint64_t)j);
            if (!(r > 0.0)) continue; /* coincident pair: no direction, w'(0) = 0 */
            double f = mj * dw * hinv4 / r; /* m_j * |grad W| / r */
            double vxij = p->vx[i] - p->vx[j], vyij = p->vy[i] - p->vy[j], vzij = p->vz[i] - p->vz[j];
            dv += f * (vxij * dx + vyij * dy + vzij * dz);
            cx += f * (vyij * dz - vzij * dy);
            cy += f * (vzij * dx - vxij * dz);
            cz += f * (vxij * dy - vyij * dx);
        }
    }
    out[0] = rho;
    out[1] = ORC_FOUR_PI_3 * sw;
    out[2] = ORC_FOUR_PI_3 * sqdw * hinv;
    out[3] = drho;
    out[4] = -dv / rho;
    out[5] = cx / rho;
    out[6] = cy / rho;
    out[7] = cz / rho;
    out[8] = 0;
    *nngb = cnt;
    *hash = hh;
}

/* out: nt x 8 doubles {rho, nw, dnw_dh, drho_dh, divv, curl_x, curl_y, curl_z} */
int orc_density_at_h(int64_t n, double box, const double *x, const double *y, const double *z,
                     const double *vx, const double *vy, const double *vz, const double *m,
                     const double *h, int64_t nt, const int64_t *targets, const uint64_t *ids,
                     double *out, int64_t *n_ngb, uint64_t *ngb_hash)
{
    orc_parts p = {n, box, x, y, z, vx, vy, vz, m};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double o[9];
        density_one(&p, i, h[i], NULL, 0, ids, o, &n_ngb[t], &ngb_hash[t]);
        memcpy(out + 8 * t, o, 8 * sizeof(double));
    }
    return 0;
}

/* Collect, in index order, every j with r_ij < R. */
static int64_t collect(const orc_parts *p, int64_t i, double R, int64_t *cand)
{
    double R2 = R * R;
    int64_t c = 0;
    for (int64_t j = 0; j < p->n; ++j) {
        double dx, dy, dz;
        if (j == i || sep2(p, i, j, &dx, &dy, &dz) < R2) cand[c++] = j;
    }
    return c;
}

/*
 * Smoothing length (Sec. 2): the root of N_w(h) = n_ngb.  N_w is non-decreasing
 * in h and strictly increasing once any neighbour lies inside h; the self term
 * alone gives (4pi/3)(8/pi) = 32/3 < n_ngb, so the root is unique.  Newton's
 * method safeguarded by bisection, to |N_w/n_ngb - 1| <= tol.  h_max caps the
 * search (returns -1 for a target whose root lies beyond it).
 * out as orc_density_at_h, evaluated at the solved h; h_out, iters per target.
 */
int orc_solve_h(int64_t n, double box, const double *x, const double *y, const double *z,
                const double *vx, const double *vy, const double *vz, const double *m,
                const double *h_guess, double n_ngb_target, double tol, double h_max,
                int64_t nt, const int64_t *targets, const uint64_t *ids,
                double *h_out, int32_t *iters, double *out, int64_t *n_ngb, uint64_t *ngb_hash)
{
    orc_parts p = {n, box, x, y, z, vx, vy, vz, m};
    int bad = 0;
#pragma omp parallel
    {
        int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 8) reduction(+ : bad)
        for (int64_t t = 0; t < nt; ++t) {
            int64_t i = targets ? targets[t] : t;
            double h = h_guess[i];
            if (!(h > 0)) h = 0.01 * box;
            double R = 2.0 * h;
            if (R > h_max) R = h_max;
            double o[9], lo = 0.0, hi;
            int64_t cnt;
            uint64_t hh;
            int64_t nc = collect(&p, i, R, cand);
            /* grow the upper bracket until N_w(hi) >= target */
            for (;;) {
                density_one(&p, i, R, cand, nc, ids, o, &cnt, &hh);
                if (o[1] >= n_ngb_target) break;
                if (R >= h_max) { R = -1; break; }
                lo = R;
                R = 2.0 * R;
                if (R > h_max) R = h_max;
                nc = collect(&p, i, R, cand);
            }
            if (R < 0) {
                h_out[t] = -1.0;
                iters[t] = -1;
                bad += 1;
                continue;
            }
            hi = R;
            if (!(h > lo && h < hi)) h = 0.5 * (lo + hi);
            int it = 0;
            for (it = 1; it <= 200; ++it) {
                density_one(&p, i, h, cand, nc, ids, o, &cnt, &hh);
                double g = o[1] - n_ngb_target;
                if (fabs(o[1] / n_ngb_target - 1.0) <= tol) break;
                if (g < 0) lo = h; else hi = h;
                double hn = (o[2] > 0) ? h - g / o[2] : 0.5 * (lo + hi);
                if (!(hn > lo && hn < hi)) hn = 0.5 * (lo + hi);
                if (hn == h) break;
                h = hn;
            }
            h_out[t] = h;
            iters[t] = it;
            memcpy(out + 8 * t, o, 8 * sizeof(double));
            n_ngb[t] = cnt;
            ngb_hash[t] = hh;
        }
        free(cand);
    }
    return bad;
}

/*
 * Quantities between the two passes (Sec. 2: every density is needed before any
 * pressure gradient can be formed):
 *   P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u),
 *   f = [1 + h/(3 rho) drho/dh]^-1   (grad-h term, Springel & Hernquist 2002),
 *   B = |div v| / (|div v| + |curl v| + 1e-4 c/h)  (Balsara 1995; 0 if the
 *       denominator vanishes; 1 when the switch is off).
 */
void orc_ghost(int64_t nt, const double *rho, const double *drho_dh, const double *divv,
               const double *curl_abs, const double *u, const double *h, double gamma, int use_balsara,
               double *P, double *c, double *f, double *B)
{
    for (int64_t t = 0; t < nt; ++t) {
        P[t] = (gamma - 1.0) * rho[t] * u[t];
        c[t] = sqrt(gamma * (gamma - 1.0) * u[t]);
        f[t] = 1.0 / (1.0 + h[t] / (3.0 * rho[t]) * drho_dh[t]);
        if (use_balsara) {
            double a = fabs(divv[t]), b = fabs(curl_abs[t]);
            double den = a + b + 1e-4 * c[t] / h[t];
            B[t] = den > 0 ? a / den : 0.0;
        } else {
            B[t] = 1.0;
        }
    }
}

/*
 * Pressure gradient and viscosity (Eq. 2, in the Gadget-2 form), for target i,
 * over every j != i with r_ij < max(h_i, h_j):
 *   dv_i/dt = -sum_j m_j [ f_i P_i/rho_i^2 grad_i W_ij(h_i) + f_j P_j/rho_j^2 grad_i W_ij(h_j)
 *                          + Pi_ij grad_i Wbar_ij ]
 *   du_i/dt =  sum_j m_j [ f_i P_i/rho_i^2 v_ij . grad_i W_ij(h_i) + 1/2 Pi_ij v_ij . grad_i Wbar_ij ]
 *   mu_ij = v_ij . r_ij / r, Pi_ij = -(alpha/2)(c_i + c_j - 3 mu_ij) mu_ij / rhobar_ij * (B_i+B_j)/2
 *   when mu_ij < 0, else 0; rhobar = (rho_i+rho_j)/2; Wbar = (W(h_i)+W(h_j))/2;
 *   vsig_i = max_j (c_i + c_j - 3 min(mu_ij, 0))  (0 without neighbours).
 * Per-particle inputs (rho, P, c, f, B) are indexed by particle, for all n.
 */
int orc_force(int64_t n, double box, const double *x, const double *y, const double *z,
              const double *vx, const double *vy, const double *vz, const double *m,
              const double *h, const double *rho, const double *P, const double *c,
              const double *f, const double *B, double alpha, int64_t nt, const int64_t *targets,
              double *ax, double *ay, double *az, double *dudt, double *vsig, int64_t *n_pairs)
{
    orc_parts p = {n, box, x, y, z, vx, vy, vz, m};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double hi = h[i], hi2 = hi * hi;
        double Ai = f[i] * P[i] / (rho[i] * rho[i]);
        double sx = 0, sy = 0, sz = 0, su = 0, vs = 0;
        int64_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx, dy, dz;
            double r2 = sep2(&p, i, j, &dx, &dy, &dz);
            double hj = h[j], hj2 = hj * hj;
            if (!(r2 < hi2 || r2 < hj2)) continue;
            ++cnt;
            double r = sqrt(r2);
            if (!(r > 0.0)) continue; /* coincident pair: no direction, w'(0) = 0 */
            double dWi = (r2 < hi2) ? orc_dw(r / hi) / (hi2 * hi2) : 0.0;
            double dWj = (r2 < hj2) ? orc_dw(r / hj) / (hj2 * hj2) : 0.0;
            double Aj = f[j] * P[j] / (rho[j] * rho[j]);
            double vxij = p.vx[i] - p.vx[j], vyij = p.vy[i] - p.vy[j], vzij = p.vz[i] - p.vz[j];
            double mu = (vxij * dx + vyij * dy + vzij * dz) / r;
            double Pi = 0.0;
            if (mu < 0.0) {
                double rhobar = 0.5 * (rho[i] + rho[j]);
                Pi = -0.5 * alpha * (c[i] + c[j] - 3.0 * mu) * mu / rhobar * 0.5 * (B[i] + B[j]);
            }
            double dWbar = 0.5 * (dWi + dWj);
            double mj = p.m[j];
            double s = mj * (Ai * dWi + Aj * dWj + Pi * dWbar) / r;
            sx -= s * dx;
            sy -= s * dy;
            sz -= s * dz;
            su += mj * mu * (Ai * dWi + 0.5 * Pi * dWbar);
            double v = c[i] + c[j] - 3.0 * (mu < 0.0 ? mu : 0.0);
            if (v > vs) vs = v;
        }
        ax[t] = sx;
        ay[t] = sy;
        az[t] = sz;
        dudt[t] = su;
        vsig[t] = vs;
        if (n_pairs) n_pairs[t] = cnt;
    }
    return 0;
}

/* ---- gravity near field (Sec. 3.2, Eq. 3) ----
 * The tree walk of Sec. 3.2 ends in two kinds of tasks: a node against the
 * multipole of a distant node, and "all particles in one node interact with all
 * particles in a nearby node".  This is the second kind, with readings (not in the
 * paper): the nodes are the cells of the periodic nc^3 grid of orc_cell_key, and a
 * particle's nearby nodes are its own cell and the 26 cells adjacent to it (each
 * cell index differs by 0 or 1 modulo nc; for nc <= 3 that is every cell); each
 * pair takes the minimal-image separation (the periodic replicas Eq. 3 mentions);
 * Eq. 3 is softened with the Plummer length eps (eps = 0 is Eq. 3 as printed, and
 * then a pair at zero separation contributes nothing):
 *   a_i   = -G sum_{j != i, near} m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2)
 *   phi_i = -G sum_{j != i, near} m_j / (|r_i - r_j|^2 + eps^2)^(1/2)
 * Every target runs over ALL j in index order and tests the pair's cells. */
static inline int cell_adjacent(int64_t a, int64_t b, int64_t nc)
{
    int64_t d = a - b;
    if (d < 0) d = -d;
    return d == 0 || d == 1 || d == nc - 1;
}

int orc_grav_p2p(int64_t n, double box, const double *x, const double *y, const double *z, const double *m,
                 int64_t nc, double G, double eps, int64_t nt, const int64_t *targets, double *ax, double *ay,
                 double *az, double *phi)
{
    if (nc < 1) return 1;
    int64_t *cx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cy = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cz = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cx || !cy || !cz) {
        free(cx);
        free(cy);
        free(cz);
        return 2;
    }
    for (int64_t j = 0; j < n; ++j) {
        const int64_t k = orc_cell_key(x[j], y[j], z[j], box, nc);
        cx[j] = k % nc;
        cy[j] = (k / nc) % nc;
        cz[j] = k / (nc * nc);
    }
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = targets ? targets[t] : t;
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (!cell_adjacent(cx[i], cx[j], nc) || !cell_adjacent(cy[i], cy[j], nc) ||
                !cell_adjacent(cz[i], cz[j], nc))
                continue;
            const double dx = min_image(x[i] - x[j], box);
            const double dy = min_image(y[i] - y[j], box);
            const double dz = min_image(z[i] - z[j], box);
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) continue; /* eps = 0, coincident particles */
            const double rinv = 1.0 / sqrt(r2);
            const double rinv3 = rinv * rinv * rinv;
            sx -= G * m[j] * dx * rinv3;
            sy -= G * m[j] * dy * rinv3;
            sz -= G * m[j] * dz * rinv3;
            sp -= G * m[j] * rinv;
        }
        ax[t] = sx;
        ay[t] = sy;
        az[t] = sz;
        phi[t] = sp;
    }
    free(cx);
    free(cy);
    free(cz);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
