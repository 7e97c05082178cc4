/*
 * fs1_ref.c -- sequential FP64 FS-1 (Liao et al., "Fast Sinkhorn I: an O(N)
 * algorithm for the Wasserstein-1 metric"), plain C99.
 *
 * TEST INFRASTRUCTURE ONLY: the CPU oracle.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg load this file's library.  It shares no
 * code, header or constant with the CUDA path.
 *
 * One solver covers:
 *   - Algorithm 1 (1D: n2 == n3 == 1), Algorithm 2 (2D: n1 fast x n2 slow,
 *     n3 == 1, the first index contiguous as in the paper's column-major
 *     flattening) and its extension to three axes that the closing remark of
 *     Section 4 states (3D: n1 fast x n2 middle x n3 slow, the separable
 *     kernel K3 (x) K2 (x) K1 applied one axis at a time);
 *   - the plain form (tau = +inf: no absorption, every factor below is lam)
 *     and the stabilised form of the Remarks in Sections 2 and 3
 *     (absorption of phi~, psi~ into A = alpha/eps, B = beta/eps when an
 *     infinity norm exceeds tau, then sweeps over the rescaled kernel
 *     K~ = diag(e^A) K diag(e^B)).
 *
 * The sweeps are the recurrences of Section 3 (eq. "recursion") and, in 2D,
 * of Section 4 (eq. "2d recursion"); in the stabilised form each factor lam
 * becomes lam e^{S_{i+1}-S_i} (forward) or lam e^{S_i-S_{i+1}} (backward) for
 * the scale field S of the output (B for K~^T phi~, A for K~ psi~), which is
 * what the Remark's replaced lines 5, 6, 10 and 11 do.  Applying the 2D kernel
 * K2 (x) K1 as a fast-axis sweep followed by a slow-axis sweep with the same
 * scale field is exact because e^S K e^-S = (e^S K2 e^-S)(e^S K1 e^-S) for the
 * separable K; the same holds axis by axis in 3D.  An axis of length 1 is the
 * identity and is skipped.
 *
 * The return value sum_ij u_i K_ij C_ij v_j is evaluated in O(N) with the
 * distance-weighted recurrences G_{k+1} = f_k (G_k + r_k),
 * H_k = b_k (H_{k+1} + s_{k+1} + x_{k+1}) (the paper writes it as an O(N^2)
 * sum; the recurrences are derived for it and pinned against the double sum).
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared fs1_ref.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { REF_OK = 0, REF_EINVAL = 1, REF_ENOMEM = 2, REF_ENUMERIC = 3, REF_ENOTCONV = 4 };

typedef struct {
    long n[3], st[3], n_all;   /* axis lengths (fast, middle, slow), strides, points */
    double lam[3];
    /* factors for the scale field S = B (K~^T phi~) and S = A (K~ psi~):
       [2 a] axis a forward, [2 a + 1] axis a backward; entry k holds the factor
       between position k and its successor along the axis */
    double *fb[6], *fa[6];
    double *eab;            /* e^{A+B} */
    double *A, *B, *ph, *ps;
    double *x, *y, *z1, *z2, *g[3];
} solver;

/* forward and backward sweep along one line (length m, stride st):
   y_k = sum_j prod(factors between j and k) x_j   (r + s of eq. "recursion") */
static void sweep_line(const double *x, double *y, long m, long st,
                       const double *ff, const double *fbk)
{
    double r = x[0];
    y[0] = r;
    for (long k = 1; k < m; ++k) {
        r = ff[(k - 1) * st] * r + x[k * st];
        y[k * st] = r;
    }
    double s = 0.0;
    for (long k = m - 2; k >= 0; --k) {
        s = fbk[k * st] * (s + x[(k + 1) * st]);
        y[k * st] += s;
    }
}

/* distance-weighted sweep: y_k = sum_j prod(factors) |k-j| x_j */
static void wsweep_line(const double *x, double *y, long m, long st,
                        const double *ff, const double *fbk)
{
    double r = x[0], G = 0.0;
    y[0] = 0.0;
    for (long k = 1; k < m; ++k) {
        G = ff[(k - 1) * st] * (G + r);
        r = ff[(k - 1) * st] * r + x[k * st];
        y[k * st] = G;
    }
    double s = 0.0, H = 0.0;
    for (long k = m - 2; k >= 0; --k) {
        H = fbk[k * st] * (H + s + x[(k + 1) * st]);
        s = fbk[k * st] * (s + x[(k + 1) * st]);
        y[k * st] += H;
    }
}

/* y = e^S K e^-S x for the separable kernel: the fast-axis sweep of every
   line along axis 0, then axis 1, then axis 2 (axes of length 1 skipped).
   weighted[a] selects the distance-weighted sweep on axis a. */
static void apply_kernel(solver *S, double *const f[6], const double *x, double *y,
                         const int weighted[3])
{
    const double *in = x;
    int todo = 0;
    for (int a = 0; a < 3; ++a) todo += S->n[a] > 1;
    if (todo == 0) {   /* a single point: K = [1] (the weighted sum is 0) */
        y[0] = weighted[0] ? 0.0 : x[0];
        return;
    }
    for (int a = 0, done = 0; a < 3; ++a) {
        if (S->n[a] <= 1) continue;
        ++done;
        double *out = (done == todo) ? y : (done == 1 ? S->z1 : S->z2);
        long m = S->n[a], st = S->st[a];
        for (long k = 0; k < S->n_all; ++k) {
            if ((k / st) % m != 0) continue;   /* k starts a line along axis a */
            if (weighted[a]) wsweep_line(in + k, out + k, m, st, f[2 * a] + k, f[2 * a + 1] + k);
            else             sweep_line(in + k, out + k, m, st, f[2 * a] + k, f[2 * a + 1] + k);
        }
        in = out;
    }
}

static void set_factors(solver *S, const double *sc, double *f[6])
{
    for (int a = 0; a < 3; ++a) {
        long m = S->n[a], st = S->st[a];
        for (long k = 0; k < S->n_all; ++k) {
            if ((k / st) % m + 1 < m) {
                double d = sc[k + st] - sc[k];
                f[2 * a][k] = S->lam[a] * exp(d);
                f[2 * a + 1][k] = S->lam[a] * exp(-d);
            } else {
                f[2 * a][k] = f[2 * a + 1][k] = 0.0;
            }
        }
    }
}

static void absorb(solver *S)
{
    /* Remark (Section 2): alpha += eps ln phi, beta += eps ln psi, phi = psi = 1;
       here A = alpha/eps, B = beta/eps. */
    for (long k = 0; k < S->n_all; ++k) {
        S->A[k] += log(S->ph[k]);
        S->B[k] += log(S->ps[k]);
        S->ph[k] = 1.0;
        S->ps[k] = 1.0;
        S->eab[k] = exp(S->A[k] + S->B[k]);
    }
    set_factors(S, S->B, S->fb);
    set_factors(S, S->A, S->fa);
}

static double maxabs(const double *x, long n)
{
    double m = 0.0;
    for (long k = 0; k < n; ++k) {
        double t = fabs(x[k]);
        if (t > m || t != t) m = t;
    }
    return m;
}

static void free_solver(solver *S)
{
    for (int q = 0; q < 6; ++q) { free(S->fb[q]); free(S->fa[q]); }
    free(S->eab); free(S->A); free(S->B); free(S->ph); free(S->ps);
    free(S->x); free(S->y); free(S->z1); free(S->z2);
    for (int a = 0; a < 3; ++a) free(S->g[a]);
}

/* axis lengths, strides and decays; an axis of length 1 needs no spacing */
static int setup(solver *S, long n1, long n2, long n3, const double h[3], double eps)
{
    long nn[3] = {n1, n2, n3};
    if (!(eps > 0.0)) return REF_EINVAL;
    S->n_all = 1;
    for (int a = 0; a < 3; ++a) {
        if (nn[a] < 1 || (nn[a] > 1 && !(h[a] > 0.0))) return REF_EINVAL;
        S->n[a] = nn[a];
        S->st[a] = S->n_all;
        S->n_all *= nn[a];
        S->lam[a] = nn[a] > 1 ? exp(-h[a] / eps) : 0.0;
    }
    return REF_OK;
}

/*
 * Solve one pair.  a, b: n1*n2*n3 histograms (fast index contiguous, then the
 * middle, then the slow one).  tau: the absorption threshold of the
 * stabilised form (pass +inf for the plain form; the stabilised form needs
 * a, b > 0).  Outputs: w (transport cost of the final iterate), iters
 * (completed iterations), err (marginal L1 error of the final iterate),
 * optional f_out, g_out (log potentials, n1*n2*n3 each).  Returns REF_OK,
 * REF_EINVAL, REF_ENOMEM or REF_ENUMERIC (a non-finite marginal error: the
 * abnormal termination of Section 5.2; iters says where).
 */
int fs1ref_solve(const double *a, const double *b, long n1, long n2, long n3,
                 double h1, double h2, double h3, double eps, double tol, long itr_max,
                 double tau, double *w, long *iters, double *err,
                 double *f_out, double *g_out)
{
    solver S;
    memset(&S, 0, sizeof S);
    const double hh[3] = {h1, h2, h3};
    if (setup(&S, n1, n2, n3, hh, eps) != REF_OK) return REF_EINVAL;
    long n = S.n_all;
    int stab = isfinite(tau) ? 1 : 0;
    if (stab)
        for (long k = 0; k < n; ++k)
            if (!(a[k] > 0.0) || !(b[k] > 0.0)) return REF_EINVAL;

    int bad = 0;
    for (int q = 0; q < 6; ++q) {
        S.fb[q] = malloc(sizeof(double) * n);
        S.fa[q] = malloc(sizeof(double) * n);
        bad |= !S.fb[q] || !S.fa[q];
    }
    double **bufs[] = {&S.eab, &S.A, &S.B, &S.ph, &S.ps, &S.x, &S.y, &S.z1, &S.z2, &S.g[0], &S.g[1], &S.g[2]};
    for (unsigned q = 0; q < sizeof bufs / sizeof bufs[0]; ++q) {
        *bufs[q] = malloc(sizeof(double) * n);
        bad |= !*bufs[q];
    }
    if (bad) { free_solver(&S); return REF_ENOMEM; }

    /* Algorithm 1 / 2, line 1: lam = e^{-h/eps}; phi = psi = 1/N */
    for (long k = 0; k < n; ++k) {
        S.A[k] = S.B[k] = 0.0;
        S.ph[k] = S.ps[k] = 1.0 / (double)n;
        S.eab[k] = 1.0;
    }
    set_factors(&S, S.B, S.fb);
    set_factors(&S, S.A, S.fa);

    static const int plain[3] = {0, 0, 0};
    long ell = 0;
    double e = 0.0;
    int status = REF_OK;
    for (;;) {
        if (stab && (maxabs(S.ph, n) > tau || maxabs(S.ps, n) > tau)) absorb(&S);
        /* r, s sweeps on phi: S.y = e^B K^T (e^A phi~) */
        for (long k = 0; k < n; ++k) S.x[k] = S.eab[k] * S.ph[k];
        apply_kernel(&S, S.fb, S.x, S.y, plain);
        /* while condition: sum_j |psi_j (K^T phi)_j - v_j| > tol */
        e = 0.0;
        for (long k = 0; k < n; ++k) e += fabs(S.ps[k] * S.y[k] - b[k]);
        if (!isfinite(e)) { status = REF_ENUMERIC; break; }
        if (ell >= itr_max || e <= tol) break;
        /* psi = v / (r + s) */
        for (long k = 0; k < n; ++k) S.ps[k] = b[k] / S.y[k];
        /* p, q sweeps on psi: S.y = e^A K (e^B psi~) */
        for (long k = 0; k < n; ++k) S.x[k] = S.eab[k] * S.ps[k];
        apply_kernel(&S, S.fa, S.x, S.y, plain);
        /* phi = u / (p + q) */
        for (long k = 0; k < n; ++k) S.ph[k] = a[k] / S.y[k];
        ++ell;
    }
    *iters = ell;
    *err = e;
    if (status == REF_OK) {
        /* return value: sum_ij u_i K_ij (sum over axes of |d_axis| h_axis) v_j
           with u = e^A phi~, v = e^B psi~: for every axis the e^A-scaled
           sweeps of e^{A+B} psi~, distance-weighted along that axis */
        for (long k = 0; k < n; ++k) S.x[k] = S.eab[k] * S.ps[k];
        double acc = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            if (S.n[ax] <= 1) continue;
            int wsel[3] = {0, 0, 0};
            wsel[ax] = 1;
            apply_kernel(&S, S.fa, S.x, S.g[ax], wsel);
            for (long k = 0; k < n; ++k) acc += S.ph[k] * hh[ax] * S.g[ax][k];
        }
        *w = acc;
        if (!isfinite(acc)) status = REF_ENUMERIC;
    } else {
        *w = NAN;
    }
    if (f_out) for (long k = 0; k < n; ++k) f_out[k] = S.A[k] + log(S.ph[k]);
    if (g_out) for (long k = 0; k < n; ++k) g_out[k] = S.B[k] + log(S.ps[k]);
    free_solver(&S);
    return status;
}

/* One product K x (x of length n1*n2*n3) with the plain recurrences; y = K x,
   distance-weighted along the axes flagged in `weighted` (bit a: axis a).
   Exposed for the recurrence-versus-dense pins. */
int fs1ref_matvec(const double *x, double *y, long n1, long n2, long n3,
                  double h1, double h2, double h3, double eps, int weighted)
{
    solver S;
    memset(&S, 0, sizeof S);
    const double hh[3] = {h1, h2, h3};
    if (setup(&S, n1, n2, n3, hh, eps) != REF_OK) return REF_EINVAL;
    long n = S.n_all;
    double *f[6];
    int bad = 0;
    for (int q = 0; q < 6; ++q) { f[q] = calloc((size_t)n, sizeof(double)); bad |= !f[q]; }
    double *zero = calloc((size_t)n, sizeof(double));
    S.z1 = malloc(sizeof(double) * n);
    S.z2 = malloc(sizeof(double) * n);
    if (bad || !zero || !S.z1 || !S.z2) {
        for (int q = 0; q < 6; ++q) free(f[q]);
        free(zero); free(S.z1); free(S.z2);
        return REF_ENOMEM;
    }
    set_factors(&S, zero, f);
    const int wsel[3] = {weighted & 1, (weighted >> 1) & 1, (weighted >> 2) & 1};
    apply_kernel(&S, f, x, y, wsel);
    for (int q = 0; q < 6; ++q) free(f[q]);
    free(zero); free(S.z1); free(S.z2);
    return REF_OK;
}
