/*
 * rp_oracle.c -- FP64 CPU oracle for the retarded scalar and vector potentials
 * of a multi-domain system (Shapira, Lomakin, Boag, Natan, "Fast calculation
 * of retarded potentials in multi-domain TDDFT", arXiv 2311.15429).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (target domain t, target node k at r_k, step l):
 *
 *   phi(r_k, l)  = sum_n sum_{k' in d_n} W(k,k') * rho_n(k', l - tau_{kk'})
 *   A(r_k, l)    = (1/c) sum_n sum_{k'} W(k,k') * J_n(k', l - tau_{kk'})
 *
 *   Eq. 2 (the Lorenz-gauge retarded integral P = int S(r', t - R/c)/R dr')
 *   summed over sub-domains (Eqs. 3-4), sampled on each domain's grid with
 *   the volume element h_n^3 (Eq. 8), where tau = R/(c dt) is the delay in
 *   steps and the source between samples is the triangle (hat) interpolant of
 *   Eq. 7:  S(t) = sum_j S_j T(t - j dt),  T(s) = max(0, 1 - |s|/dt).
 *   Evaluated at the retarded time this is
 *       S(l - tau) = (1 - w) S_{l-m} + w S_{l-m-1},   m = floor(tau), w = tau - m,
 *   which is the same number as sum_m G_m S_{l-m} with the space-time
 *   sampled Green's function of Eq. 11, G_m = h^3 T(m dt - R/c)/R (Eq. 12).
 *
 *   Weights:  W = h_n^3 / R for R > 0.
 *             At R = 0 (target node == source node of its own domain) the
 *             1/R singularity is replaced by its average over the cell, a
 *             cube of side h:  h^3 <1/R>_cube = C h^2 with
 *             C = 3 ln(2 + sqrt 3) - pi/2, taken at lag 0.  The paper defers
 *             the self-point treatment to a "smoothed Green's function"
 *             (Sec. III, after Eq. 6); the cube average is the reading used.
 *
 *   The charge q_e of the paper's four-vector source (Sec. II, before Eq. 2)
 *   is not applied: the caller multiplies by q_e = -1 if wanted.
 *
 * History: the caller passes, per domain n, the samples for steps
 * hist_first[n] .. hist_first[n] + hist_len[n] - 1 (rpo_eval: one window
 * for all domains), each sample laid out as [4][N_n] (rho, Jx, Jy, Jz;
 * x fastest within a field).  A sample outside the window is an error,
 * except that with `clamp` a sample older than the window equals its first
 * sample -- the paper's S(t <= 0) = S(0) of Eqs. 7 and 9.
 *
 * Arithmetic: every sample is promoted to double; each of the four sums is
 * Neumaier-compensated.  c may be +INFINITY (instantaneous limit: tau = 0).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define RPO_OK 0
#define RPO_ERR_HISTORY 1
#define RPO_ERR_ARG 2
#define RPO_ERR_COINCIDENT 3

/* Neumaier (improved Kahan) accumulator. */
typedef struct {
    double s, comp;
} rpo_acc;

static void acc_add(rpo_acc *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->comp += (a->s - t) + x;
    else
        a->comp += (x - t) + a->s;
    a->s = t;
}

static double acc_value(const rpo_acc *a) { return a->s + a->comp; }

/* The cube average of 1/|r| over a cube of side 1 centred on the origin. */
static double cube_average_constant(void)
{
    return 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * M_PI;
}

/* Sample (field f, node q) of domain n at time index j, promoted to double;
 * domain n's stored window starts at time index first[n] and holds len[n]
 * samples. */
static int fetch(const void *const *hist, int is_f64, const long long *first, const int *len, int clamp,
                 int n, long long N, int f, long long q, long long j, double *out)
{
    const long long hist_first = first[n];
    const int hist_len = len[n];
    long long idx = j - hist_first;
    if (idx < 0) {
        if (!clamp)
            return RPO_ERR_HISTORY;
        idx = 0;
    }
    if (idx >= hist_len)
        return RPO_ERR_HISTORY;
    long long off = (idx * 4 + f) * N + q;
    if (is_f64)
        *out = ((const double *)hist[n])[off];
    else
        *out = (double)((const float *)hist[n])[off];
    return RPO_OK;
}

/*
 * rpo_eval_windows -- retarded phi and A at a list of nodes of one target domain.
 *
 *   ndom            number of domains
 *   origin[3*n]     position of node (0,0,0) of domain n
 *   nn[3*n]         grid points (nx, ny, nz) of domain n; node id = x + nx*(y + ny*z)
 *   h[n]            grid spacing of domain n
 *   hist[n]         samples of domain n, [hist_len[n]][4][N_n], float or double
 *   hist_is_f64     nonzero: hist holds doubles
 *   hist_first[n]   time index of hist[n][0]
 *   hist_len[n]     number of stored samples of domain n
 *   c, dt           speed of light and time step (atomic units)
 *   clamp           nonzero: samples before hist_first equal hist_first's
 *   target, step    target domain and the time index l evaluated
 *   npts, nodes     node ids in the target domain
 *   out[4*npts]     phi, Ax, Ay, Az per node
 *
 * Returns RPO_OK, RPO_ERR_HISTORY (a sample outside the stored window),
 * RPO_ERR_ARG, or RPO_ERR_COINCIDENT (nodes of two different domains at the
 * same place, where 1/R has no defined value).
 */
int rpo_eval_windows(int ndom, const double *origin, const int *nn, const double *h,
                     const void *const *hist, int hist_is_f64, const long long *hist_first,
                     const int *hist_len, double c, double dt, int clamp,
                     int target, long long step, int npts, const long long *nodes, double *out)
{
    if (ndom <= 0 || target < 0 || target >= ndom || npts < 0 || !(dt > 0.0) || !(c > 0.0))
        return RPO_ERR_ARG;
    for (int n = 0; n < ndom; ++n)
        if (hist_len[n] <= 0)
            return RPO_ERR_ARG;
    const double C = cube_average_constant();
    const int tx = nn[3 * target + 0], ty = nn[3 * target + 1], tz = nn[3 * target + 2];
    const long long Nt = (long long)tx * ty * tz;

    for (int p = 0; p < npts; ++p) {
        long long k = nodes[p];
        if (k < 0 || k >= Nt)
            return RPO_ERR_ARG;
        int ix = (int)(k % tx), iy = (int)((k / tx) % ty), iz = (int)(k / ((long long)tx * ty));
        double rx = origin[3 * target + 0] + h[target] * ix;
        double ry = origin[3 * target + 1] + h[target] * iy;
        double rz = origin[3 * target + 2] + h[target] * iz;

        rpo_acc acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

        for (int n = 0; n < ndom; ++n) {
            const int sx = nn[3 * n + 0], sy = nn[3 * n + 1], sz = nn[3 * n + 2];
            const long long Ns = (long long)sx * sy * sz;
            const double hs = h[n];
            const double vol = hs * hs * hs;
            for (long long q = 0; q < Ns; ++q) {
                int jx = (int)(q % sx), jy = (int)((q / sx) % sy), jz = (int)(q / ((long long)sx * sy));
                double s[4];
                if (n == target && q == k) {
                    /* the node's own cell: cube-averaged 1/R, no delay */
                    double w0 = C * hs * hs;
                    for (int f = 0; f < 4; ++f) {
                        int e = fetch(hist, hist_is_f64, hist_first, hist_len, clamp, n, Ns, f, q, step, &s[f]);
                        if (e)
                            return e;
                        acc_add(&acc[f], w0 * s[f]);
                    }
                    continue;
                }
                double dx = rx - (origin[3 * n + 0] + hs * jx);
                double dy = ry - (origin[3 * n + 1] + hs * jy);
                double dz = rz - (origin[3 * n + 2] + hs * jz);
                double R = sqrt(dx * dx + dy * dy + dz * dz);
                if (R == 0.0)
                    return RPO_ERR_COINCIDENT;
                double tau = R / (c * dt);      /* delay in steps */
                double m = floor(tau);
                double w = tau - m;             /* weight of the older sample */
                long long j0 = (long long)step - (long long)m;
                for (int f = 0; f < 4; ++f) {
                    double a, b = 0.0;
                    int e = fetch(hist, hist_is_f64, hist_first, hist_len, clamp, n, Ns, f, q, j0, &a);
                    if (e)
                        return e;
                    if (w > 0.0) {
                        e = fetch(hist, hist_is_f64, hist_first, hist_len, clamp, n, Ns, f, q, j0 - 1, &b);
                        if (e)
                            return e;
                    }
                    double sr = (1.0 - w) * a + w * b;
                    acc_add(&acc[f], vol * sr / R);
                }
            }
        }
        out[4 * p + 0] = acc_value(&acc[0]);
        for (int f = 1; f < 4; ++f)
            out[4 * p + f] = acc_value(&acc[f]) / c;
    }
    return RPO_OK;
}

/*
 * rpo_eval -- rpo_eval_windows with one stored window for every domain:
 * samples hist_first .. hist_first + hist_len - 1.
 */
int rpo_eval(int ndom, const double *origin, const int *nn, const double *h,
             const void *const *hist, int hist_is_f64, int hist_first, int hist_len,
             double c, double dt, int clamp,
             int target, int step, int npts, const long long *nodes, double *out)
{
    if (ndom <= 0 || ndom > 4096)
        return RPO_ERR_ARG;
    long long first[4096];
    int len[4096];
    for (int n = 0; n < ndom; ++n) {
        first[n] = hist_first;
        len[n] = hist_len;
    }
    return rpo_eval_windows(ndom, origin, nn, h, hist, hist_is_f64, first, len, c, dt, clamp, target,
                            step, npts, nodes, out);
}

/*
 * rpo_eval_positions -- the same retarded sums at arbitrary points (not grid
 * nodes): every node of every domain is a source with weight h_n^3 / R and
 * the hat-interpolated sample at the retarded time (Eqs. 2, 7, 8).  There is
 * no self cell; a point on a source node is RPO_ERR_COINCIDENT.
 *
 *   pos[3*p]        position of point p (bohr)
 *   out[4*npos]     phi, Ax, Ay, Az per point (A with the 1/c factor)
 *
 * Other arguments as for rpo_eval.
 */
int rpo_eval_positions(int ndom, const double *origin, const int *nn, const double *h,
                       const void *const *hist, int hist_is_f64, int hist_first_in, int hist_len_in,
                       double c, double dt, int clamp, int step, int npos, const double *pos, double *out)
{
    if (ndom <= 0 || ndom > 4096 || npos < 0 || hist_len_in <= 0 || !(dt > 0.0) || !(c > 0.0))
        return RPO_ERR_ARG;
    long long hist_first[4096];
    int hist_len[4096];
    for (int n = 0; n < ndom; ++n) {
        hist_first[n] = hist_first_in;
        hist_len[n] = hist_len_in;
    }
    for (int p = 0; p < npos; ++p) {
        const double rx = pos[3 * p + 0], ry = pos[3 * p + 1], rz = pos[3 * p + 2];
        rpo_acc acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (int n = 0; n < ndom; ++n) {
            const int sx = nn[3 * n + 0], sy = nn[3 * n + 1], sz = nn[3 * n + 2];
            const long long Ns = (long long)sx * sy * sz;
            const double hs = h[n];
            const double vol = hs * hs * hs;
            for (long long q = 0; q < Ns; ++q) {
                int jx = (int)(q % sx), jy = (int)((q / sx) % sy), jz = (int)(q / ((long long)sx * sy));
                double dx = rx - (origin[3 * n + 0] + hs * jx);
                double dy = ry - (origin[3 * n + 1] + hs * jy);
                double dz = rz - (origin[3 * n + 2] + hs * jz);
                double R = sqrt(dx * dx + dy * dy + dz * dz);
                if (R == 0.0)
                    return RPO_ERR_COINCIDENT;
                double tau = R / (c * dt);
                double m = floor(tau);
                double w = tau - m;
                long long j0 = (long long)step - (long long)m;
                for (int f = 0; f < 4; ++f) {
                    double a, b = 0.0;
                    int e = fetch(hist, hist_is_f64, hist_first, hist_len, clamp, n, Ns, f, q, j0, &a);
                    if (e)
                        return e;
                    if (w > 0.0) {
                        e = fetch(hist, hist_is_f64, hist_first, hist_len, clamp, n, Ns, f, q, j0 - 1, &b);
                        if (e)
                            return e;
                    }
                    acc_add(&acc[f], vol * ((1.0 - w) * a + w * b) / R);
                }
            }
        }
        out[4 * p + 0] = acc_value(&acc[0]);
        for (int f = 1; f < 4; ++f)
            out[4 * p + f] = acc_value(&acc[f]) / c;
    }
    return RPO_OK;
}

/* The value of C used above, for the tests that pin it. */
double rpo_cube_average_constant(void) { return cube_average_constant(); }
