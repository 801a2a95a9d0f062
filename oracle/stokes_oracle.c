/*
 * stokes_oracle.c -- FP64 CPU oracle for the periodized 2-D Stokes layer-potential sum.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code with the CUDA library; the two see the same
 * inputs only.
 *
 * What it computes is the plain discrete definition, written as a double loop:
 *
 *   For every target node i and every image m in {-1, 0, +1} (shift m*(d,0)):
 *   - single-layer (vesicle) source j, skipped when j lies on the target's own
 *     curve and m = 0:   add S(x_i, y_j + m d) w_j f_j        (stokeslet, Eq. (S))
 *   - double-layer (wall) source j, skipped when j = i and m = 0:
 *                         add D(x_i, y_j + m d) w_j tau_j      (stresslet, Eq. (D))
 *   The image range is the near-image sum of Eq. (Dnr) and Eq. (utotrep).
 *   Then at a wall node add the Nystrom diagonal -kappa/(2 pi) t t^T w tau
 *   (Sec. 2.3) and jump * tau (jump = -1/2 gives the interior limit, Eq. (JR)),
 *   and at a vesicle node add the Kress product-quadrature self term of the
 *   single layer (the log-split periodic rule the paper uses for the self
 *   interaction, Sec. 3.2).
 *
 * Accumulation is FP64, per target in the order images -1, 0, +1 (outer) and
 * sources in ascending index (inner), then the self terms.  OpenMP splits the
 * target loop only, so each target's summation order does not depend on the
 * thread count.
 *
 * Kress rule for a closed curve sampled at n (even) equispaced parameter
 * values t_k = 2 pi k / n, with speed s_k = |x'(t_k)| = w_k n / (2 pi):
 *   u_i = 1/(4 pi mu) sum_k [ -1/2 R_{(i-k) mod n} I
 *                            + (2 pi / n) ( -1/2 L_ik I + M_ik ) ] s_k f_k
 *   R_j  = -(4 pi / n) sum_{p=1}^{n/2-1} cos(2 pi p j / n) / p - (4 pi / n^2) (-1)^j
 *          (weights of int_0^{2pi} log(4 sin^2((t - tau)/2)) phi(tau) dtau)
 *   L_ik = log(|x_i - x_k|^2 / (4 sin^2(pi (i - k) / n))),  L_ii = log(s_i^2)
 *   M_ik = r r^T / r^2,                                      M_ii = t_i t_i^T
 * i.e. log(1/r) = -1/2 log(4 sin^2) - 1/2 L, the first part integrated by the
 * product rule and the smooth remainder by the trapezoid rule.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

enum { ORA_KIND_DLP = 0, ORA_KIND_SLP = 1 };

/* Stokeslet S(x, y) applied to f, Eq. (S): (1/(4 pi mu)) (log(1/r) f + r (r.f)/r^2). */
static void ora_stokeslet_apply(double r1, double r2, double mu, double f1, double f2,
                                double *u1, double *u2)
{
    double rr = r1 * r1 + r2 * r2;
    double lg = log(1.0 / sqrt(rr));
    double rf = (r1 * f1 + r2 * f2) / rr;
    double c = 1.0 / (4.0 * ORA_PI * mu);
    *u1 = c * (lg * f1 + r1 * rf);
    *u2 = c * (lg * f2 + r2 * rf);
}

/* Stresslet D(x, y) applied to tau, Eq. (D): (1/pi) r (r.tau) (r.n_y) / r^4. */
static void ora_stresslet_apply(double r1, double r2, double n1, double n2, double t1, double t2,
                                double *u1, double *u2)
{
    double rr = r1 * r1 + r2 * r2;
    double rn = r1 * n1 + r2 * n2;
    double rt = r1 * t1 + r2 * t2;
    double c = rn * rt / (ORA_PI * rr * rr);
    *u1 = c * r1;
    *u2 = c * r2;
}

/* The full 2x2 tensors, for the pointwise tests. */
void ora_stokeslet_tensor(double x1, double x2, double y1, double y2, double mu, double *S)
{
    double e1[2], e2[2];
    ora_stokeslet_apply(x1 - y1, x2 - y2, mu, 1.0, 0.0, &e1[0], &e1[1]);
    ora_stokeslet_apply(x1 - y1, x2 - y2, mu, 0.0, 1.0, &e2[0], &e2[1]);
    S[0] = e1[0]; S[1] = e2[0]; S[2] = e1[1]; S[3] = e2[1];
}

void ora_stresslet_tensor(double x1, double x2, double y1, double y2, double n1, double n2,
                          double *D)
{
    double e1[2], e2[2];
    ora_stresslet_apply(x1 - y1, x2 - y2, n1, n2, 1.0, 0.0, &e1[0], &e1[1]);
    ora_stresslet_apply(x1 - y1, x2 - y2, n1, n2, 0.0, 1.0, &e2[0], &e2[1]);
    D[0] = e1[0]; D[1] = e2[0]; D[2] = e1[1]; D[3] = e2[1];
}

/* Kress weights R_j, j = 0..n-1, from their defining cosine sum. */
int ora_kress_weights(int n, double *R)
{
    if (n < 2 || (n & 1)) return -4;
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int p = 1; p <= n / 2 - 1; ++p)
            acc += cos(2.0 * ORA_PI * (double)p * (double)j / (double)n) / (double)p;
        R[j] = -(4.0 * ORA_PI / n) * acc - (4.0 * ORA_PI / ((double)n * n)) * ((j & 1) ? -1.0 : 1.0);
    }
    return 0;
}

typedef struct {
    int n_nodes, n_curves;
    const int *off, *kind;
    const double *x, *w, *nrm, *kap;
    double period, mu;
    const double *slp, *dlp;
    int *curve_of;   /* node -> curve */
    int *dens_of;    /* node -> row in slp or dlp density */
    double **R;      /* Kress weights per curve (NULL for walls) */
} ora_geom;

static int ora_geom_init(ora_geom *g)
{
    g->curve_of = (int *)malloc(sizeof(int) * (size_t)(g->n_nodes > 0 ? g->n_nodes : 1));
    g->dens_of = (int *)malloc(sizeof(int) * (size_t)(g->n_nodes > 0 ? g->n_nodes : 1));
    g->R = (double **)calloc((size_t)(g->n_curves > 0 ? g->n_curves : 1), sizeof(double *));
    if (!g->curve_of || !g->dens_of || !g->R) return -8;
    int ns = 0, nd = 0;
    for (int c = 0; c < g->n_curves; ++c) {
        int n = g->off[c + 1] - g->off[c];
        for (int i = g->off[c]; i < g->off[c + 1]; ++i) {
            g->curve_of[i] = c;
            g->dens_of[i] = (g->kind[c] == ORA_KIND_SLP) ? ns++ : nd++;
        }
        if (g->kind[c] == ORA_KIND_SLP) {
            g->R[c] = (double *)malloc(sizeof(double) * (size_t)n);
            if (!g->R[c]) return -8;
            int st = ora_kress_weights(n, g->R[c]);
            if (st) return st;
        }
    }
    return 0;
}

static void ora_geom_free(ora_geom *g)
{
    if (g->R) for (int c = 0; c < g->n_curves; ++c) free(g->R[c]);
    free(g->R); free(g->curve_of); free(g->dens_of);
}

/* Sum over all sources and images at point (px, py); own curve / own node per the skip rules.
 * self_node < 0 means a free target: nothing is skipped. */
static void ora_pair_sum(const ora_geom *g, double px, double py, int self_node, double *o1, double *o2)
{
    int self_curve = self_node >= 0 ? g->curve_of[self_node] : -1;
    int m_lo = g->period != 0.0 ? -1 : 0, m_hi = g->period != 0.0 ? 1 : 0;
    double u1 = 0.0, u2 = 0.0;
    for (int m = m_lo; m <= m_hi; ++m) {
        double sx = (double)m * g->period;
        for (int j = 0; j < g->n_nodes; ++j) {
            int c = g->curve_of[j];
            double r1 = px - (g->x[2 * j] + sx), r2 = py - g->x[2 * j + 1];
            double a1, a2;
            if (g->kind[c] == ORA_KIND_SLP) {
                if (m == 0 && c == self_curve) continue;
                const double *f = g->slp + 2 * g->dens_of[j];
                ora_stokeslet_apply(r1, r2, g->mu, g->w[j] * f[0], g->w[j] * f[1], &a1, &a2);
            } else {
                if (m == 0 && j == self_node) continue;
                const double *t = g->dlp + 2 * g->dens_of[j];
                ora_stresslet_apply(r1, r2, g->nrm[2 * j], g->nrm[2 * j + 1],
                                    g->w[j] * t[0], g->w[j] * t[1], &a1, &a2);
            }
            u1 += a1;
            u2 += a2;
        }
    }
    *o1 = u1;
    *o2 = u2;
}

/* Kress self term of the single layer at node i of a vesicle curve. */
static void ora_kress_self(const ora_geom *g, int i, double *o1, double *o2)
{
    int c = g->curve_of[i];
    int b = g->off[c], n = g->off[c + 1] - b, a = i - b;
    const double *R = g->R[c];
    double h = 2.0 * ORA_PI / n;
    double cmu = 1.0 / (4.0 * ORA_PI * g->mu);
    double u1 = 0.0, u2 = 0.0;
    for (int k = 0; k < n; ++k) {
        int j = b + k;
        double s = g->w[j] / h;                      /* speed |x'(t_k)| */
        const double *f = g->slp + 2 * g->dens_of[j];
        double L, M11, M12, M22;
        if (k == a) {
            L = log(s * s);
            double t1 = -g->nrm[2 * j + 1], t2 = g->nrm[2 * j];  /* unit tangent */
            M11 = t1 * t1; M12 = t1 * t2; M22 = t2 * t2;
        } else {
            double r1 = g->x[2 * i] - g->x[2 * j], r2 = g->x[2 * i + 1] - g->x[2 * j + 1];
            double rr = r1 * r1 + r2 * r2;
            double sn = sin(ORA_PI * (double)(a - k) / n);
            L = log(rr / (4.0 * sn * sn));
            M11 = r1 * r1 / rr; M12 = r1 * r2 / rr; M22 = r2 * r2 / rr;
        }
        int dj = a - k; if (dj < 0) dj += n;
        double diag = -0.5 * R[dj] + h * (-0.5 * L);
        double g1 = cmu * s * f[0], g2 = cmu * s * f[1];
        u1 += diag * g1 + h * (M11 * g1 + M12 * g2);
        u2 += diag * g2 + h * (M12 * g1 + M22 * g2);
    }
    *o1 = u1;
    *o2 = u2;
}

static int ora_check(int n_nodes, int n_curves, const int *off, const int *kind)
{
    if (n_nodes < 0 || n_curves < 0 || !off || (n_curves > 0 && !kind)) return -1;
    if (off[0] != 0 || off[n_curves] != n_nodes) return -1;
    for (int c = 0; c < n_curves; ++c) {
        int n = off[c + 1] - off[c];
        if (n <= 0) return -1;
        if (kind[c] != ORA_KIND_DLP && kind[c] != ORA_KIND_SLP) return -1;
        if (kind[c] == ORA_KIND_SLP && (n & 1)) return -4;
    }
    return 0;
}

/*
 * Sum at the geometry's own nodes (with self terms).
 * nodes, normals: (N, 2) row-major; weights, curvature: (N,).
 * slp_density: rows for the single-layer nodes in node order; dlp_density likewise.
 * sel: NULL for all N targets, else n_sel node indices; out is (n_sel or N, 2).
 * period = 0 switches the images off (m = 0 only).
 */
int ora_sum(int n_nodes, int n_curves, const int *curve_offset, const int *curve_kind,
            const double *nodes, const double *weights, const double *normals,
            const double *curvature, double period, double mu,
            const double *slp_density, const double *dlp_density, double jump,
            int n_sel, const int *sel, double *out, int n_threads)
{
    int st = ora_check(n_nodes, n_curves, curve_offset, curve_kind);
    if (st) return st;
    ora_geom g = {n_nodes, n_curves, curve_offset, curve_kind, nodes, weights, normals, curvature,
                  period, mu, slp_density, dlp_density, NULL, NULL, NULL};
    st = ora_geom_init(&g);
    if (st) { ora_geom_free(&g); return st; }
    int nt = sel ? n_sel : n_nodes;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int t = 0; t < nt; ++t) {
        int i = sel ? sel[t] : t;
        double u1, u2;
        ora_pair_sum(&g, nodes[2 * i], nodes[2 * i + 1], i, &u1, &u2);
        int c = g.curve_of[i];
        if (curve_kind[c] == ORA_KIND_DLP) {
            const double *tau = dlp_density + 2 * g.dens_of[i];
            double t1 = -normals[2 * i + 1], t2 = normals[2 * i];
            double k = -curvature[i] / (2.0 * ORA_PI) * weights[i] * (t1 * tau[0] + t2 * tau[1]);
            u1 += k * t1 + jump * tau[0];
            u2 += k * t2 + jump * tau[1];
        } else {
            double s1, s2;
            ora_kress_self(&g, i, &s1, &s2);
            u1 += s1;
            u2 += s2;
        }
        out[2 * t] = u1;
        out[2 * t + 1] = u2;
    }
    ora_geom_free(&g);
    return 0;
}

/* Sum at free points (plain trapezoid rule over every source and image, no self terms). */
int ora_sum_free(int n_nodes, int n_curves, const int *curve_offset, const int *curve_kind,
                 const double *nodes, const double *weights, const double *normals,
                 double period, double mu, const double *slp_density, const double *dlp_density,
                 int n_targets, const double *targets, double *out, int n_threads)
{
    int st = ora_check(n_nodes, n_curves, curve_offset, curve_kind);
    if (st) return st;
    ora_geom g = {n_nodes, n_curves, curve_offset, curve_kind, nodes, weights, normals, NULL,
                  period, mu, slp_density, dlp_density, NULL, NULL, NULL};
    st = ora_geom_init(&g);
    if (st) { ora_geom_free(&g); return st; }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int t = 0; t < n_targets; ++t) {
        double u1, u2;
        ora_pair_sum(&g, targets[2 * t], targets[2 * t + 1], -1, &u1, &u2);
        out[2 * t] = u1;
        out[2 * t + 1] = u2;
    }
    ora_geom_free(&g);
    return 0;
}

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
