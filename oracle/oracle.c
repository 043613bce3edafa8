/*
 * PAID oracle: a plain, slow, FP64 CPU implementation of the adaptive
 * cubature of the Brillouin-zone bubble integrals.
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA library:
 * rule nodes and weights are recomputed here from the closed form, and every
 * formula is written out directly from its definition.
 *
 * What it computes (paper section / equation / algorithm):
 *   - dispersion of the t-t' square-lattice Hubbard model      (Sec. 2)
 *   - orthonormal lattice form factors f_n                      (Sec. 2)
 *   - the bubble integrals, in the Matsubara-summed temperature form
 *       ph: (1/(2pi)^2) Int f_l(k) f_m(k+q) [nF(e(k+q)) - nF(e(k))] / (e(k) - e(k+q))
 *       pp: (1/(2pi)^2) Int f_l(k) f_m(q-k) [1 - nF(e(k)) - nF(e(q-k))] / (e(k) + e(q-k))
 *     with the analytic limit at a vanishing denominator
 *     (the momentum integrals of Eq. chi_pp / chi_ph, Sec. 2)
 *   - the nested Clenshaw-Curtis pair Q_N, Q_2N with err = |Q_N - Q_2N|,
 *     the N nodes being a subset of the 2N nodes              (Sec. 3)
 *   - greedy adaptive integration with 2x2 subdivision of the
 *     largest-error sub-domain                       (Algorithm 1, Sec. 3;
 *                                       4-way split as in Algorithm 2)
 *   - the group form: one heap and one error sum over all (l, m) pairs of
 *     a (kind, q)                         (Algorithm 2, global error, Sec. 4)
 *   - per-integral independence: integrals run in parallel over OpenMP
 *     threads, one integral per task (Sec. 4 distributes independent work
 *     in the same way).
 *
 * Pins (tests that tie this file to something other than itself):
 *   cc rule          closed-form weights vs. moment equations, N=4 values
 *   region rule      monomial exactness up to degree 9 (fine), 5 (coarse)
 *   form factors     Gram matrix = identity at q=0, = trig shift matrix at q
 *   kernel F         high-precision direct evaluation of the definition
 *   full integrals   dense periodic trapezoid and Gauss-Legendre brute force,
 *                    C4v and q -> -q symmetries, nesting identity, dn/dmu
 *   adaptive driver  a hand-stepped greedy on tiny budgets
 *   group driver     one pair = Algorithm 1 exactly; a hand-stepped group
 *                    greedy on tiny budgets; brute-force values per pair
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { ORC_PH = 0, ORC_PP = 1, ORC_MONOMIAL = 2, ORC_OVERLAP = 3, ORC_FLOW_PH = 4, ORC_FLOW_PP = 5 };
enum { ORC_CONVERGED = 0, ORC_BUDGET = 1, ORC_NONFINITE = 2 };
#define ORC_MAX_LEVEL 29
#define ORC_MAX_RULE_N 16

/* ------------------------------------------------------------------------
 * Clenshaw-Curtis rule on [-1,1] with N intervals (N+1 nodes, N even):
 *   x_j = cos(j pi / N),
 *   w_j = (c_j / N) [1 - sum_{k=1}^{N/2} b_k cos(2 k j pi / N) / (4k^2 - 1)],
 *   c_0 = c_N = 1, else 2;  b_{N/2} = 1, else 2.
 * Sec. 3 (closed form from the review the paper cites for CCQ).
 * Returns 0 on success, -1 for an invalid N.
 * ---------------------------------------------------------------------- */
int oracle_cc_rule(int N, double* nodes, double* weights)
{
    if (N < 2 || N % 2 != 0 || N > 2 * ORC_MAX_RULE_N) return -1;
    for (int j = 0; j <= N; ++j) {
        double cj = (j == 0 || j == N) ? 1.0 : 2.0;
        double s = 0.0;
        for (int k = 1; k <= N / 2; ++k) {
            double bk = (k == N / 2) ? 1.0 : 2.0;
            s += bk * cos(2.0 * k * j * ORC_PI / N) / (4.0 * k * k - 1.0);
        }
        nodes[j] = cos(j * ORC_PI / N);
        weights[j] = cj / N * (1.0 - s);
    }
    return 0;
}

/* Dispersion, Sec. 2:  e(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky - mu */
double oracle_dispersion(double kx, double ky, double t, double tp, double mu)
{
    return -2.0 * t * (cos(kx) + cos(ky)) - 4.0 * tp * cos(kx) * cos(ky) - mu;
}

/* Orthonormal form factors, Sec. 2 ("complete set of orthonormal functions").
 * Orthonormal under (1/(2pi)^2) Int over [-pi,pi]^2.
 *   shell 0 (on-site):            f0 = 1
 *   shell 1 (nearest neighbour):  f1 = cx + cy, f2 = cx - cy,
 *                                 f3 = sqrt2 sx, f4 = sqrt2 sy
 *   shell 2 (diagonal neighbour): f5 = 2 cx cy, f6 = 2 sx sy,
 *                                 f7 = 2 sx cy, f8 = 2 cx sy            */
double oracle_form_factor(int n, double kx, double ky)
{
    switch (n) {
    case 0: return 1.0;
    case 1: return cos(kx) + cos(ky);
    case 2: return cos(kx) - cos(ky);
    case 3: return sqrt(2.0) * sin(kx);
    case 4: return sqrt(2.0) * sin(ky);
    case 5: return 2.0 * cos(kx) * cos(ky);
    case 6: return 2.0 * sin(kx) * sin(ky);
    case 7: return 2.0 * sin(kx) * cos(ky);
    case 8: return 2.0 * cos(kx) * sin(ky);
    default: return NAN;
    }
}

/* Fermi function nF(e) = 1 / (exp(e/T) + 1). */
static double fermi(double e, double T) { return 1.0 / (exp(e / T) + 1.0); }

/* nF(b) - nF(a) without cancellation, from exact identities only:
 *   |a - b| / 2T < 1:  nF(b) - nF(a) = (tanh(a/2T) - tanh(b/2T)) / 2
 *                      = sinh((a-b)/2T) / (2 cosh(a/2T) cosh(b/2T));
 *   a, b both < 0:     nF(e) = 1 - nF(-e) gives nF(-a) - nF(-b);
 *   otherwise the direct difference (no cancellation there). */
static double fermi_diff(double b, double a, double T)
{
    double d = (a - b) / (2.0 * T);   /* exact difference first */
    if (fabs(d) < 1.0)
        return sinh(d) / (2.0 * cosh(a / (2.0 * T)) * cosh(b / (2.0 * T)));
    if (a < 0.0 && b < 0.0)
        return fermi(-a, T) - fermi(-b, T);
    return fermi(b, T) - fermi(a, T);
}

/* -nF'(e) = 1 / (4T cosh^2(e/2T)). */
static double minus_fermi_prime(double e, double T)
{
    double c = cosh(e / (2.0 * T));
    return 1.0 / (4.0 * T * c * c);
}

/* Particle-hole kernel [nF(e2) - nF(e1)] / (e1 - e2), and -nF'(e1) at e1 = e2
 * (the ph bubble of Eq. chi_ph after the Matsubara sum). */
double oracle_kernel_ph(double e1, double e2, double T)
{
    if (e1 == e2) return minus_fermi_prime(e1, T);
    return fermi_diff(e2, e1, T) / (e1 - e2);
}

/* Particle-particle kernel [1 - nF(e1) - nF(e2)] / (e1 + e2), and its limit
 * -nF'(e1) at e1 + e2 = 0 (the pp bubble of Eq. chi_pp after the Matsubara
 * sum).  1 - nF(e1) - nF(e2) = nF(-e2) - nF(e1) exactly. */
double oracle_kernel_pp(double e1, double e2, double T)
{
    if (e1 == -e2) return minus_fermi_prime(e1, T);
    return fermi_diff(-e2, e1, T) / (e1 + e2);
}

/* ---------------------------------------------------------------------------
 * Omega-regulated flow kernels: the inner frequency integrals of Eqs. chi_ph
 * and chi_pp (Sec. 2) with G(k) = theta(k0) / (i k0 - e(k)),
 * theta(k0) = k0^2 / (k0^2 + Omega^2), at zero temperature with measure
 * dk0 / 2pi, differentiated with respect to Omega (the dot of the flow).
 *
 * Derivation (written out here because the paper only states that these
 * integrals can be done analytically): theta^2 = 1 - 2 Omega^2 / (k0^2 + Omega^2)
 * + Omega^4 / (k0^2 + Omega^2)^2, and 1 / ((i k0 - e1)(i k0 - e2)) =
 * [1/(i k0 - e1) - 1/(i k0 - e2)] / (e1 - e2).  Each piece reduces to
 *   int dk0/2pi 1 / ((k0^2 + a^2)(k0^2 + b^2)) = 1 / (2 a b (a + b))
 * and its a-derivative (the odd parts of 1/(i k0 - e) integrate to zero), so
 * the ph integral is the divided difference [H(e1) - H(e2)] / (e1 - e2) of
 *   H(e) = int dk0/2pi theta^2 / (i k0 - e) = -e (2|e| + Omega) / (4 (|e| + Omega)^2),
 * and its Omega derivative the divided difference of
 *   Hdot(e) = e (3|e| + Omega) / (4 (|e| + Omega)^3).
 * pp: theta is even and -i k0 - e2 = -(i k0 + e2), so the pp integral is minus
 * the ph one at (e1, -e2).
 *
 * For e >= 0 with u = e + Omega, Hdot = (3/u - 5 Omega/u^2 + 2 Omega^2/u^3) / 4,
 * and Hdot is odd, so for energies of one sign the divided difference is that
 * of the three powers of 1/u at u_k = |e_k| + Omega, each by its exact identity
 *   D[1/u] = -1/(u1 u2),  D[1/u^2] = -(u1 + u2)/(u1 u2)^2,
 *   D[1/u^3] = -(u1^2 + u1 u2 + u2^2)/(u1 u2)^3;
 * for opposite signs the two values of Hdot have opposite signs and the
 * difference is taken directly. */
static double flow_hdot(double e, double W)
{
    const double a = fabs(e), u = a + W;
    return e * (3.0 * a + W) / (4.0 * u * u * u);
}

double oracle_kernel_flow_ph(double e1, double e2, double W)
{
    if ((e1 >= 0.0) != (e2 >= 0.0))
        return (flow_hdot(e1, W) - flow_hdot(e2, W)) / (e1 - e2);
    const double u1 = fabs(e1) + W, u2 = fabs(e2) + W, p = u1 * u2;
    const double d1 = -1.0 / p;
    const double d2 = -(u1 + u2) / (p * p);
    const double d3 = -(u1 * u1 + u1 * u2 + u2 * u2) / (p * p * p);
    return 0.25 * (3.0 * d1 - 5.0 * W * d2 + 2.0 * W * W * d3);
}

double oracle_kernel_flow_pp(double e1, double e2, double W)
{
    return -oracle_kernel_flow_ph(e1, -e2, W);
}

/* One integral's parameters. */
typedef struct {
    int kind;           /* ORC_PH, ORC_PP, ORC_MONOMIAL, ORC_OVERLAP, ORC_FLOW_PH, ORC_FLOW_PP */
    double qx, qy;      /* transfer momentum */
    int l, m;           /* form-factor indices (MONOMIAL: exponents a, b) */
    double T;           /* temperature (flow kinds: the regulator scale Omega) */
    double t, tp, mu;   /* lattice parameters */
} orc_integral;

/* The integrand at k = (kx, ky), including the 1/(2pi)^2 prefactor.
 *   ph:       f_l(k) f_m(k+q) F_ph(e(k), e(k+q))         (Eq. chi_ph, T form)
 *   pp:       f_l(k) f_m(q-k) F_pp(e(k), e(q-k))         (Eq. chi_pp, T form)
 *   overlap:  f_l(k) f_m(k+q)                             (F = 1)
 *   monomial: (kx/pi)^l (ky/pi)^m                         (rule test)
 *   flow ph:  f_l(k) f_m(k) Fdot_ph(e(k + q/2), e(k - q/2))  (Eq. chi_ph, Omega form)
 *   flow pp:  f_l(k) f_m(k) Fdot_pp(e(q/2 + k), e(q/2 - k))  (Eq. chi_pp, Omega form) */
static double integrand(const orc_integral* p, double kx, double ky)
{
    const double pref = 1.0 / (4.0 * ORC_PI * ORC_PI);
    double e1, e2;
    switch (p->kind) {
    case ORC_PH:
        e1 = oracle_dispersion(kx, ky, p->t, p->tp, p->mu);
        e2 = oracle_dispersion(kx + p->qx, ky + p->qy, p->t, p->tp, p->mu);
        return pref * oracle_form_factor(p->l, kx, ky)
                    * oracle_form_factor(p->m, kx + p->qx, ky + p->qy)
                    * oracle_kernel_ph(e1, e2, p->T);
    case ORC_PP:
        e1 = oracle_dispersion(kx, ky, p->t, p->tp, p->mu);
        e2 = oracle_dispersion(p->qx - kx, p->qy - ky, p->t, p->tp, p->mu);
        return pref * oracle_form_factor(p->l, kx, ky)
                    * oracle_form_factor(p->m, p->qx - kx, p->qy - ky)
                    * oracle_kernel_pp(e1, e2, p->T);
    case ORC_OVERLAP:
        return pref * oracle_form_factor(p->l, kx, ky)
                    * oracle_form_factor(p->m, kx + p->qx, ky + p->qy);
    case ORC_MONOMIAL:
        return pref * pow(kx / ORC_PI, p->l) * pow(ky / ORC_PI, p->m);
    case ORC_FLOW_PH:   /* symmetric routing: k +- l/2, both form factors at k */
    case ORC_FLOW_PP:   /* e(l/2 - k) = e(k - l/2): the dispersion is even */
        e1 = oracle_dispersion(kx + 0.5 * p->qx, ky + 0.5 * p->qy, p->t, p->tp, p->mu);
        e2 = oracle_dispersion(kx - 0.5 * p->qx, ky - 0.5 * p->qy, p->t, p->tp, p->mu);
        return pref * oracle_form_factor(p->l, kx, ky) * oracle_form_factor(p->m, kx, ky)
                    * (p->kind == ORC_FLOW_PH ? oracle_kernel_flow_ph(e1, e2, p->T)
                                              : oracle_kernel_flow_pp(e1, e2, p->T));
    default:
        return NAN;
    }
}

/* Exported for tests: one integrand value. */
double oracle_integrand_point(int kind, double qx, double qy, int l, int m,
                              double T, double t, double tp, double mu,
                              double kx, double ky)
{
    orc_integral p = {kind, qx, qy, l, m, T, t, tp, mu};
    return integrand(&p, kx, ky);
}

/* ------------------------------------------------------------------------
 * Region rule, Sec. 3.  A region is the dyadic square of level L with
 * integer corner (ix, iy) in [0, 2^L)^2:
 *   [-pi + ix h, -pi + (ix+1) h] x [-pi + iy h, -pi + (iy+1) h],  h = 2pi/2^L.
 * Q_2N is the tensor product of the 2N-interval CC rule (fine), Q_N that of
 * the N-interval rule (coarse), whose nodes are the even-indexed fine nodes.
 * ---------------------------------------------------------------------- */
typedef struct {
    int N;
    double xf[2 * ORC_MAX_RULE_N + 1], wf[2 * ORC_MAX_RULE_N + 1]; /* 2N intervals */
    double xc[ORC_MAX_RULE_N + 1], wc[ORC_MAX_RULE_N + 1];         /* N intervals */
} orc_rule;

static int make_rule(int N, orc_rule* r)
{
    if (N < 2 || N % 2 != 0 || N > ORC_MAX_RULE_N) return -1;
    r->N = N;
    if (oracle_cc_rule(2 * N, r->xf, r->wf)) return -1;
    if (oracle_cc_rule(N, r->xc, r->wc)) return -1;
    return 0;
}

static void region_rule(const orc_integral* p, const orc_rule* r,
                        int L, int64_t ix, int64_t iy, double* qN, double* q2N)
{
    double h = 2.0 * ORC_PI / ldexp(1.0, L);
    double x0 = -ORC_PI + (double)ix * h, y0 = -ORC_PI + (double)iy * h;
    int nf = 2 * r->N;
    double sf = 0.0, sc = 0.0;
    for (int i = 0; i <= nf; ++i) {
        double kx = x0 + 0.5 * h * (1.0 + r->xf[i]);
        for (int j = 0; j <= nf; ++j) {
            double ky = y0 + 0.5 * h * (1.0 + r->xf[j]);
            double g = integrand(p, kx, ky);
            sf += r->wf[i] * r->wf[j] * g;
            if (i % 2 == 0 && j % 2 == 0)
                sc += r->wc[i / 2] * r->wc[j / 2] * g;
        }
    }
    double jac = 0.25 * h * h;  /* (h/2)^2 */
    *q2N = jac * sf;
    *qN = jac * sc;
}

/* Exported for tests: Q_N and Q_2N of one region. */
int oracle_region_eval(int kind, double qx, double qy, int l, int m, double T,
                       double t, double tp, double mu, int rule_n,
                       int L, int64_t ix, int64_t iy, double* qN, double* q2N)
{
    orc_rule r;
    if (make_rule(rule_n, &r)) return -1;
    orc_integral p = {kind, qx, qy, l, m, T, t, tp, mu};
    region_rule(&p, &r, L, ix, iy, qN, q2N);
    return 0;
}

/* ------------------------------------------------------------------------
 * Task record and max-heap keyed by err (Sec. 4: task {id, domain, val_N,
 * val_2N, err}; the container is a heap on err).  Ties: smaller level, then
 * smaller ix, then smaller iy first.
 * ---------------------------------------------------------------------- */
typedef struct {
    int L;
    int64_t ix, iy;
    double valN, val2N, err;
} orc_task;

static int task_before(const orc_task* a, const orc_task* b)
{
    if (a->err != b->err) return a->err > b->err;
    if (a->L != b->L) return a->L < b->L;
    if (a->ix != b->ix) return a->ix < b->ix;
    return a->iy < b->iy;
}

static void heap_push(orc_task* h, int64_t* n, orc_task t)
{
    int64_t i = (*n)++;
    h[i] = t;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!task_before(&h[i], &h[par])) break;
        orc_task tmp = h[i]; h[i] = h[par]; h[par] = tmp;
        i = par;
    }
}

static orc_task heap_pop(orc_task* h, int64_t* n)
{
    orc_task top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t a = 2 * i + 1, b = 2 * i + 2, best = i;
        if (a < *n && task_before(&h[a], &h[best])) best = a;
        if (b < *n && task_before(&h[b], &h[best])) best = b;
        if (best == i) break;
        orc_task tmp = h[i]; h[i] = h[best]; h[best] = tmp;
        i = best;
    }
    return top;
}

static orc_task make_task(const orc_integral* p, const orc_rule* r, int L, int64_t ix, int64_t iy)
{
    orc_task t;
    t.L = L; t.ix = ix; t.iy = iy;
    region_rule(p, r, L, ix, iy, &t.valN, &t.val2N);
    t.err = fabs(t.valN - t.val2N);
    return t;
}

static void exact_sums(const orc_task* h, int64_t n, double* V, double* E)
{
    double v = 0.0, e = 0.0;
    for (int64_t i = 0; i < n; ++i) { v += h[i].val2N; e += h[i].err; }
    *V = v; *E = e;
}

/* ------------------------------------------------------------------------
 * Algorithm 1 (Sec. 3) for one integral, with the 4-way split of
 * Algorithm 2 and the initial partition a uniform grid of level L0:
 *   evaluate every initial region, push it (Listing 1);
 *   while E > max(abs_tol, rel_tol |V|):
 *       take the region with the largest err (extract-max),
 *       split it into 4 (Listing 3), evaluate the children,
 *       E += sum(child err) - parent err, V likewise (Listing 4),
 *       push the children;
 *   return V = sum of Q_2N over the leaves (Listing 5), E, leaf count.
 * A split is made only while the leaf count stays <= max_regions and the
 * region is above the deepest level; otherwise the status is BUDGET.
 * E and V are recomputed exactly from the leaves every 1024 splits and at
 * the end, so that no rounding drift accumulates.
 * If `trace` is non-NULL the final leaves are copied to it (up to trace_cap).
 * ---------------------------------------------------------------------- */
static int adaptive_one(const orc_integral* p, const orc_rule* r, int L0,
                        double rel_tol, double abs_tol, int64_t max_regions,
                        double* value, double* error, int64_t* regions,
                        orc_task* trace, int64_t trace_cap, int64_t* trace_n)
{
    int64_t n0 = (int64_t)1 << (2 * L0);
    int64_t cap = max_regions > n0 ? max_regions : n0;
    orc_task* heap = (orc_task*)malloc((size_t)(cap + 4) * sizeof(orc_task));
    if (!heap) return -1;
    int64_t n = 0;
    int64_t side = (int64_t)1 << L0;
    for (int64_t ix = 0; ix < side; ++ix)
        for (int64_t iy = 0; iy < side; ++iy)
            heap_push(heap, &n, make_task(p, r, L0, ix, iy));
    double V, E;
    exact_sums(heap, n, &V, &E);
    int status = ORC_CONVERGED;
    int64_t splits = 0;
    for (;;) {
        if (!isfinite(V) || !isfinite(E)) { status = ORC_NONFINITE; break; }
        double tol = fmax(abs_tol, rel_tol * fabs(V));
        if (E <= tol) { status = ORC_CONVERGED; break; }
        if (n + 3 > max_regions || heap[0].L >= ORC_MAX_LEVEL) { status = ORC_BUDGET; break; }
        orc_task par = heap_pop(heap, &n);
        E -= par.err;
        V -= par.val2N;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                orc_task c = make_task(p, r, par.L + 1, 2 * par.ix + a, 2 * par.iy + b);
                E += c.err;
                V += c.val2N;
                heap_push(heap, &n, c);
            }
        if (++splits % 1024 == 0) exact_sums(heap, n, &V, &E);
    }
    exact_sums(heap, n, &V, &E);
    if (!isfinite(V) || !isfinite(E)) status = ORC_NONFINITE;
    *value = V; *error = E; *regions = n;
    if (trace) {
        int64_t k = n < trace_cap ? n : trace_cap;
        memcpy(trace, heap, (size_t)k * sizeof(orc_task));
        *trace_n = n;
    }
    free(heap);
    return status;
}

/* ------------------------------------------------------------------------
 * Batch entry point: integrals are (q, pair) with idx = iq * npairs + ip.
 * Each integral is independent; they are spread over `nthreads` OpenMP
 * threads with dynamic scheduling (0 = all available threads).
 * Returns 0, or -1 for an invalid argument.
 * ---------------------------------------------------------------------- */
int oracle_integrate_batch(int kind, int nq, const double* q, int npairs, const int32_t* lm,
                           double T, double t, double tp, double mu,
                           double rel_tol, double abs_tol, int64_t max_regions,
                           int rule_n, int init_level, int nthreads,
                           double* values, double* errors, int64_t* regions, int32_t* status)
{
    orc_rule r;
    if (make_rule(rule_n, &r)) return -1;
    if (nq < 0 || npairs < 0 || init_level < 0 || init_level > 12) return -1;
    int64_t n = (int64_t)nq * npairs;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int64_t iq = i / npairs, ip = i % npairs;
        orc_integral p = {kind, q[2 * iq], q[2 * iq + 1], lm[2 * ip], lm[2 * ip + 1],
                          T, t, tp, mu};
        int st = adaptive_one(&p, &r, init_level, rel_tol, abs_tol, max_regions,
                              &values[i], &errors[i], &regions[i], NULL, 0, NULL);
        status[i] = st < 0 ? ORC_NONFINITE : st;
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------------
 * Algorithm 2 (Sec. 4) for one group: all (l, m) pairs of one (kind, q).
 * Every pair keeps its own partition (a uniform level-L0 grid at the start,
 * Listing 1), but the tasks of all pairs sit in one max-heap and one error
 * sum decides when the group is done (the global error of Sec. 4: the sum of
 * the pairs' absolute errors, without the coupling norms):
 *   while E_g = sum_c E_c > max(abs_tol, rel_tol sum_c |V_c|):
 *       take the task (pair, region) with the largest err over the group,
 *       split it into 4, evaluate the children for that pair,
 *       update that pair's E_c, V_c, push the children.
 * With rel_tol = 0 the test is the paper's absolute E_g < eps.  A split is
 * made only while the popped pair stays within max_regions leaves and the
 * region is above the deepest level; otherwise the group stops with BUDGET.
 * Ties in the heap: larger err, then smaller pair index, level, ix, iy.
 * Sums are recomputed exactly from the leaves every 1024 splits and at the
 * end.  Every pair of the group gets the group's status.
 * ---------------------------------------------------------------------- */
typedef struct {
    orc_task t;
    int c;              /* pair index within the group */
} orc_gtask;

static int gtask_before(const orc_gtask* a, const orc_gtask* b)
{
    if (a->t.err != b->t.err) return a->t.err > b->t.err;
    if (a->c != b->c) return a->c < b->c;
    return task_before(&a->t, &b->t);
}

static void gheap_push(orc_gtask* h, int64_t* n, orc_gtask t)
{
    int64_t i = (*n)++;
    h[i] = t;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!gtask_before(&h[i], &h[par])) break;
        orc_gtask tmp = h[i]; h[i] = h[par]; h[par] = tmp;
        i = par;
    }
}

static orc_gtask gheap_pop(orc_gtask* h, int64_t* n)
{
    orc_gtask top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t a = 2 * i + 1, b = 2 * i + 2, best = i;
        if (a < *n && gtask_before(&h[a], &h[best])) best = a;
        if (b < *n && gtask_before(&h[b], &h[best])) best = b;
        if (best == i) break;
        orc_gtask tmp = h[i]; h[i] = h[best]; h[best] = tmp;
        i = best;
    }
    return top;
}

static void group_exact_sums(const orc_gtask* h, int64_t n, int P, double* V, double* E)
{
    for (int c = 0; c < P; ++c) { V[c] = 0.0; E[c] = 0.0; }
    for (int64_t i = 0; i < n; ++i) { V[h[i].c] += h[i].t.val2N; E[h[i].c] += h[i].t.err; }
}

static int adaptive_group(const orc_integral* pairs, int P, const orc_rule* r, int L0,
                          double rel_tol, double abs_tol, int64_t max_regions,
                          double* V, double* E, int64_t* leaves)
{
    int64_t n0 = (int64_t)1 << (2 * L0);
    int64_t hcap = (int64_t)P * n0 * 4 + 4;   /* grows by doubling */
    orc_gtask* heap = (orc_gtask*)malloc((size_t)hcap * sizeof(orc_gtask));
    if (!heap) return -1;
    int64_t n = 0;
    int64_t side = (int64_t)1 << L0;
    for (int c = 0; c < P; ++c) {
        leaves[c] = n0;
        for (int64_t ix = 0; ix < side; ++ix)
            for (int64_t iy = 0; iy < side; ++iy) {
                orc_gtask g = {make_task(&pairs[c], r, L0, ix, iy), c};
                gheap_push(heap, &n, g);
            }
    }
    group_exact_sums(heap, n, P, V, E);
    int status = ORC_CONVERGED;
    int64_t splits = 0;
    for (;;) {
        double Eg = 0.0, Vabs = 0.0;
        int finite = 1;
        for (int c = 0; c < P; ++c) {
            if (!isfinite(V[c]) || !isfinite(E[c])) finite = 0;
            Eg += E[c];
            Vabs += fabs(V[c]);
        }
        if (!finite) { status = ORC_NONFINITE; break; }
        if (Eg <= fmax(abs_tol, rel_tol * Vabs)) { status = ORC_CONVERGED; break; }
        const orc_gtask* top = &heap[0];
        if (leaves[top->c] + 3 > max_regions || top->t.L >= ORC_MAX_LEVEL) {
            status = ORC_BUDGET;
            break;
        }
        if (n + 4 > hcap) {
            orc_gtask* h2 = (orc_gtask*)realloc(heap, (size_t)(2 * hcap) * sizeof(orc_gtask));
            if (!h2) { free(heap); return -1; }
            heap = h2;
            hcap *= 2;
        }
        orc_gtask par = gheap_pop(heap, &n);
        int c = par.c;
        E[c] -= par.t.err;
        V[c] -= par.t.val2N;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                orc_gtask ch = {make_task(&pairs[c], r, par.t.L + 1, 2 * par.t.ix + a,
                                          2 * par.t.iy + b), c};
                E[c] += ch.t.err;
                V[c] += ch.t.val2N;
                gheap_push(heap, &n, ch);
            }
        leaves[c] += 3;
        if (++splits % 1024 == 0) group_exact_sums(heap, n, P, V, E);
    }
    group_exact_sums(heap, n, P, V, E);
    for (int c = 0; c < P; ++c)
        if (!isfinite(V[c]) || !isfinite(E[c])) status = ORC_NONFINITE;
    free(heap);
    return status;
}

/* Batch entry point of Algorithm 2: one group per q row, its pairs the
 * batch's (l, m) list; outputs in the batch order idx = iq * npairs + ip
 * (every pair's own V_c, E_c and leaf count; the group's status).  Groups run
 * in parallel over `nthreads` OpenMP threads.  Returns 0, or -1 for an
 * invalid argument. */
int oracle_integrate_group_global(int kind, int nq, const double* q, int npairs, const int32_t* lm,
                                  double T, double t, double tp, double mu,
                                  double rel_tol, double abs_tol, int64_t max_regions,
                                  int rule_n, int init_level, int nthreads,
                                  double* values, double* errors, int64_t* regions,
                                  int32_t* status)
{
    orc_rule r;
    if (make_rule(rule_n, &r)) return -1;
    if (nq < 0 || npairs < 1 || init_level < 0 || init_level > 12) return -1;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int iq = 0; iq < nq; ++iq) {
        orc_integral* pairs = (orc_integral*)malloc((size_t)npairs * sizeof(orc_integral));
        int st = -1;
        int64_t o = (int64_t)iq * npairs;
        if (pairs) {
            for (int c = 0; c < npairs; ++c) {
                orc_integral p = {kind, q[2 * iq], q[2 * iq + 1], lm[2 * c], lm[2 * c + 1],
                                  T, t, tp, mu};
                pairs[c] = p;
            }
            st = adaptive_group(pairs, npairs, &r, init_level, rel_tol, abs_tol, max_regions,
                                &values[o], &errors[o], &regions[o]);
            free(pairs);
        }
        for (int c = 0; c < npairs; ++c) status[o + c] = st < 0 ? ORC_NONFINITE : st;
    }
    (void)nthreads;
    return 0;
}

/* Same, over a flat list of integrals with per-integral kind, q, (l, m) and T
 * (used for mixed samples).  Returns 0 or -1. */
int oracle_integrate_list(int64_t n, const int32_t* kind, const double* q, const int32_t* lm,
                          const double* T, double t, double tp, double mu,
                          double rel_tol, double abs_tol, int64_t max_regions,
                          int rule_n, int init_level, int nthreads,
                          double* values, double* errors, int64_t* regions, int32_t* status)
{
    orc_rule r;
    if (make_rule(rule_n, &r)) return -1;
    if (n < 0 || init_level < 0 || init_level > 12) return -1;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t i = 0; i < n; ++i) {
        orc_integral p = {kind[i], q[2 * i], q[2 * i + 1], lm[2 * i], lm[2 * i + 1],
                          T[i], t, tp, mu};
        int st = adaptive_one(&p, &r, init_level, rel_tol, abs_tol, max_regions,
                              &values[i], &errors[i], &regions[i], NULL, 0, NULL);
        status[i] = st < 0 ? ORC_NONFINITE : st;
    }
    (void)nthreads;
    return 0;
}

/* One integral with its final leaf set: keys (L, ix, iy) and (Q_N, Q_2N, err)
 * per leaf, for the driver pin and for the proposal's training targets.
 * Returns the status, or -1. */
int oracle_integrate_trace(int kind, double qx, double qy, int l, int m, double T,
                           double t, double tp, double mu,
                           double rel_tol, double abs_tol, int64_t max_regions,
                           int rule_n, int init_level,
                           double* value, double* error, int64_t* nleaves,
                           int64_t trace_cap, int32_t* leaf_level, int64_t* leaf_ix,
                           int64_t* leaf_iy, double* leaf_valN, double* leaf_val2N,
                           double* leaf_err)
{
    orc_rule r;
    if (make_rule(rule_n, &r)) return -1;
    orc_integral p = {kind, qx, qy, l, m, T, t, tp, mu};
    orc_task* tr = (orc_task*)malloc((size_t)(trace_cap > 0 ? trace_cap : 1) * sizeof(orc_task));
    if (!tr) return -1;
    int64_t tn = 0;
    int st = adaptive_one(&p, &r, init_level, rel_tol, abs_tol, max_regions,
                          value, error, nleaves, tr, trace_cap, &tn);
    int64_t k = tn < trace_cap ? tn : trace_cap;
    for (int64_t i = 0; i < k; ++i) {
        leaf_level[i] = tr[i].L; leaf_ix[i] = tr[i].ix; leaf_iy[i] = tr[i].iy;
        leaf_valN[i] = tr[i].valN; leaf_val2N[i] = tr[i].val2N; leaf_err[i] = tr[i].err;
    }
    free(tr);
    return st;
}

/* The integral by its definition on a dense periodic grid: the M x M
 * trapezoid rule over [-pi, pi)^2 (spectrally convergent for these analytic
 * periodic integrands; converged values are independent of any adaptive
 * partition).  Used to decide which side is wrong when two adaptive results
 * disagree beyond their tolerances.  Returns the value (NAN for M < 1). */
double oracle_trapezoid(int kind, double qx, double qy, int l, int m, double T,
                        double t, double tp, double mu, int M, int nthreads)
{
    if (M < 1) return NAN;
    orc_integral p = {kind, qx, qy, l, m, T, t, tp, mu};
    double h = 2.0 * ORC_PI / M;
    double total = 0.0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) reduction(+ : total) num_threads(nt)
#endif
    for (int i = 0; i < M; ++i) {
        double row = 0.0;
        for (int j = 0; j < M; ++j)
            row += integrand(&p, -ORC_PI + i * h, -ORC_PI + j * h);
        total += row;
    }
    (void)nthreads;
    return total * h * h;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
