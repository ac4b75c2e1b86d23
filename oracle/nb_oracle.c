/*
 * FP64 CPU oracle for the Ahmad-Cohen regular force, its time derivative,
 * the neighbour list and the Hermite predictor (Nitadori & Aarseth 2012,
 * "Accelerating NBODY6 with Graphics Processing Units").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Every routine is written straight from the definitions in the paper:
 *   - neighbour criterion: Sec. 3.2, the two displayed criteria
 *     (|R_ij| < h_i, and the velocity form min(|R_ij|, |R_ij + dtR_i V_ij|) < h_i);
 *   - regular force, regular jerk and neighbour list: Sec. 3.3, step (vi);
 *   - irregular force and jerk (sum over the list only): Sec. 3.3, step (iv);
 *   - prediction of the j-particles to the block time: Sec. 3.3, step (iii)
 *     (the paper names the step but prints no formula; the Hermite scheme of
 *     Sec. 2 carries a and da/dt, so the prediction is the Taylor polynomial in
 *     those: positions to third order in dt, velocities to second order).
 * G = 1 throughout.  All arithmetic is IEEE double; no reassociation flags.
 *
 * Readings where the paper is silent (each also listed with the design notes):
 *   - a pair with R_min exactly equal to h_i is not a neighbour and goes into
 *     the regular sum (the force case reads "> h_i", the list "< h_i"; strict
 *     "<" for the list makes the two sums a partition of all j != i);
 *   - self is excluded by index, never by distance;
 *   - the list is ascending in j; at most `cap` entries are stored (the lowest
 *     `cap` indices), the count returned is the true count and the overflow
 *     flag is set when the count exceeds `cap`;
 *   - dtr == NULL selects the plain criterion |R_ij| < h_i;
 *   - a coincident pair j != i (|R_ij| = 0) that is not a neighbour has no
 *     defined force; the oracle reports ORC_ERR_COINCIDENT for it.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_COINCIDENT (-2)

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Neighbour test of Sec. 3.2: R_min < h_i, with R_min = |R| for the plain
 * criterion and min(|R|, |R + dtr V|) for the velocity criterion. */
static int is_neighbour(const double R[3], const double V[3], double h_i,
                        const double *dtr_i)
{
    double rmin = sqrt(dot3(R, R));
    if (dtr_i) {
        double Rp[3];
        for (int k = 0; k < 3; k++) Rp[k] = R[k] + (*dtr_i) * V[k];
        double rp = sqrt(dot3(Rp, Rp));
        if (rp < rmin) rmin = rp;
    }
    return rmin < h_i;
}

/* One term of the force sum and of the jerk sum (Sec. 3.3, (iv) and (vi)):
 *   F += m_j R / |R|^3
 *   J += m_j [ V / |R|^3 - 3 (R.V) R / |R|^5 ]
 * pot += m_j / |R| (the potential, same sign as the GPU listing of App. B). */
static void add_term(const double R[3], const double V[3], double m_j,
                     double F[3], double J[3], double *pot)
{
    double r2 = dot3(R, R);
    double r = sqrt(r2);
    double r3 = r2 * r;
    double r5 = r3 * r2;
    double rv = dot3(R, V);
    for (int k = 0; k < 3; k++) {
        F[k] += m_j * R[k] / r3;
        J[k] += m_j * (V[k] / r3 - 3.0 * rv * R[k] / r5);
    }
    if (pot) *pot += m_j / r;
}

/*
 * Prediction of all j-particles to the block time t (Sec. 3.3, step (iii)):
 *   dt = t - t0_j
 *   x  = x0 + v0 dt + a0 dt^2/2 + adot0 dt^3/6
 *   v  = v0 + a0 dt + adot0 dt^2/2
 * Arrays are [n][3] row-major (x of particle j at 3j..3j+2).
 */
int orc_predict(int64_t n, const double *x0, const double *v0,
                const double *a0, const double *adot0, const double *t0,
                double t, double *x, double *v)
{
    if (n < 0 || (n > 0 && (!x0 || !v0 || !a0 || !adot0 || !t0 || !x || !v)))
        return ORC_ERR_ARG;
    for (int64_t j = 0; j < n; j++) {
        double dt = t - t0[j];
        double dt2 = dt * dt;
        double dt3 = dt2 * dt;
        for (int k = 0; k < 3; k++) {
            int64_t q = 3 * j + k;
            x[q] = x0[q] + v0[q] * dt + a0[q] * dt2 / 2.0 + adot0[q] * dt3 / 6.0;
            v[q] = v0[q] + a0[q] * dt + adot0[q] * dt2 / 2.0;
        }
    }
    return ORC_OK;
}

/*
 * Regular force, regular jerk and neighbour list of each active particle
 * (Sec. 3.3, step (vi)), for active particles act[0..n_act) indexing the
 * predicted set x, v, m of n particles.
 *   h[i]    neighbour radius of active particle i (>= 0)
 *   dtr     NULL, or dtr[i] = regular step of active particle i (Sec. 3.2)
 *   F, J    [n_act][3] outputs;  pot (nullable) [n_act]
 *   nnb     [n_act] true neighbour count
 *   list    [n_act][cap] ascending neighbour indices (first min(nnb,cap))
 *   ovf     [n_act] 1 when nnb > cap
 * nthreads <= 0 uses one thread per host core (OpenMP over active particles).
 */
int orc_regular(int64_t n, const double *x, const double *v, const double *m,
                int32_t n_act, const int32_t *act, const double *h,
                const double *dtr, int32_t cap, double *F, double *J,
                double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf,
                int nthreads)
{
    if (n < 0 || n_act < 0 || cap < 0) return ORC_ERR_ARG;
    if (n_act > 0 && (!x || !v || !m || !act || !h || !F || !J || !nnb || !ovf))
        return ORC_ERR_ARG;
    if (n_act > 0 && cap > 0 && !list) return ORC_ERR_ARG;
    for (int32_t a = 0; a < n_act; a++)
        if (act[a] < 0 || act[a] >= n) return ORC_ERR_ARG;
    int status = ORC_OK;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int32_t a = 0; a < n_act; a++) {
        int64_t i = act[a];
        double Fi[3] = {0, 0, 0}, Ji[3] = {0, 0, 0}, pi = 0.0;
        int32_t count = 0;
        const double *dtr_i = dtr ? &dtr[a] : NULL;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double R[3], V[3];
            for (int k = 0; k < 3; k++) {
                R[k] = x[3 * j + k] - x[3 * i + k];
                V[k] = v[3 * j + k] - v[3 * i + k];
            }
            if (is_neighbour(R, V, h[a], dtr_i)) {
                if (count < cap) list[(int64_t)a * cap + count] = (int32_t)j;
                count++;
            } else {
                if (dot3(R, R) == 0.0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    status = ORC_ERR_COINCIDENT;
                    continue;
                }
                add_term(R, V, m[j], Fi, Ji, pot ? &pi : NULL);
            }
        }
        for (int k = 0; k < 3; k++) {
            F[3 * (int64_t)a + k] = Fi[k];
            J[3 * (int64_t)a + k] = Ji[k];
        }
        if (pot) pot[a] = pi;
        nnb[a] = count;
        ovf[a] = count > cap ? 1 : 0;
    }
    return status;
}

/*
 * Irregular force and jerk (Sec. 3.3, step (iv)): the same pair terms summed
 * over the neighbour set L_i only (the full set, not clipped to any capacity),
 * with L_i decided by the same criterion as in orc_regular.
 */
int orc_irregular(int64_t n, const double *x, const double *v, const double *m,
                  int32_t n_act, const int32_t *act, const double *h,
                  const double *dtr, double *F, double *J, int nthreads)
{
    if (n < 0 || n_act < 0) return ORC_ERR_ARG;
    if (n_act > 0 && (!x || !v || !m || !act || !h || !F || !J)) return ORC_ERR_ARG;
    for (int32_t a = 0; a < n_act; a++)
        if (act[a] < 0 || act[a] >= n) return ORC_ERR_ARG;
    int status = ORC_OK;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int32_t a = 0; a < n_act; a++) {
        int64_t i = act[a];
        double Fi[3] = {0, 0, 0}, Ji[3] = {0, 0, 0};
        const double *dtr_i = dtr ? &dtr[a] : NULL;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double R[3], V[3];
            for (int k = 0; k < 3; k++) {
                R[k] = x[3 * j + k] - x[3 * i + k];
                V[k] = v[3 * j + k] - v[3 * i + k];
            }
            if (!is_neighbour(R, V, h[a], dtr_i)) continue;
            if (dot3(R, R) == 0.0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                status = ORC_ERR_COINCIDENT;
                continue;
            }
            add_term(R, V, m[j], Fi, Ji, NULL);
        }
        for (int k = 0; k < 3; k++) {
            F[3 * (int64_t)a + k] = Fi[k];
            J[3 * (int64_t)a + k] = Ji[k];
        }
    }
    return status;
}

/*
 * Full direct sum with no neighbour split: F and J summed over every j != i
 * (the total force that the regular and irregular parts add up to, Sec. 1 and
 * Sec. 3.3).  pot (nullable) receives sum m_j/|R|.
 */
int orc_full(int64_t n, const double *x, const double *v, const double *m,
             int32_t n_act, const int32_t *act, double *F, double *J,
             double *pot, int nthreads)
{
    if (n < 0 || n_act < 0) return ORC_ERR_ARG;
    if (n_act > 0 && (!x || !v || !m || !act || !F || !J)) return ORC_ERR_ARG;
    for (int32_t a = 0; a < n_act; a++)
        if (act[a] < 0 || act[a] >= n) return ORC_ERR_ARG;
    int status = ORC_OK;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int32_t a = 0; a < n_act; a++) {
        int64_t i = act[a];
        double Fi[3] = {0, 0, 0}, Ji[3] = {0, 0, 0}, pi = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double R[3], V[3];
            for (int k = 0; k < 3; k++) {
                R[k] = x[3 * j + k] - x[3 * i + k];
                V[k] = v[3 * j + k] - v[3 * i + k];
            }
            if (dot3(R, R) == 0.0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                status = ORC_ERR_COINCIDENT;
                continue;
            }
            add_term(R, V, m[j], Fi, Ji, pot ? &pi : NULL);
        }
        for (int k = 0; k < 3; k++) {
            F[3 * (int64_t)a + k] = Fi[k];
            J[3 * (int64_t)a + k] = Ji[k];
        }
        if (pot) pot[a] = pi;
    }
    return status;
}

/*
 * Conditioning of the regular sums: for each active particle, the sums over
 * its regular set (the j that orc_regular sums) of the lengths of the
 * individual force and jerk terms,
 *   SF_i = sum_j |m_j R / |R|^3|,
 *   SJ_i = sum_j |m_j [ V / |R|^3 - 3 (R.V) R / |R|^5 ]|.
 * SF_i / |F_i| and SJ_i / |J_i| are the condition numbers of the two sums: a
 * sum whose terms each carry a relative rounding error e has an absolute
 * error of at most e SF_i (e SJ_i), however much the terms cancel.  Used to
 * state the tolerance of working-precision pair terms on rows whose regular
 * force or jerk nearly cancels.
 */
int orc_regular_mag(int64_t n, const double *x, const double *v, const double *m,
                    int32_t n_act, const int32_t *act, const double *h,
                    const double *dtr, double *SF, double *SJ, int nthreads)
{
    if (n < 0 || n_act < 0) return ORC_ERR_ARG;
    if (n_act > 0 && (!x || !v || !m || !act || !h || !SF || !SJ)) return ORC_ERR_ARG;
    for (int32_t a = 0; a < n_act; a++)
        if (act[a] < 0 || act[a] >= n) return ORC_ERR_ARG;
    int status = ORC_OK;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int32_t a = 0; a < n_act; a++) {
        int64_t i = act[a];
        double sf = 0.0, sj = 0.0;
        const double *dtr_i = dtr ? &dtr[a] : NULL;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double R[3], V[3];
            for (int k = 0; k < 3; k++) {
                R[k] = x[3 * j + k] - x[3 * i + k];
                V[k] = v[3 * j + k] - v[3 * i + k];
            }
            if (is_neighbour(R, V, h[a], dtr_i)) continue;
            double r2 = dot3(R, R);
            if (r2 == 0.0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                status = ORC_ERR_COINCIDENT;
                continue;
            }
            double r = sqrt(r2);
            double fJ[3];
            for (int k = 0; k < 3; k++) fJ[k] = m[j] * (V[k] / (r2 * r) - 3.0 * dot3(R, V) * R[k] / (r2 * r2 * r));
            sf += m[j] / r2;   /* |m R / |R|^3| */
            sj += sqrt(dot3(fJ, fJ));
        }
        SF[a] = sf;
        SJ[a] = sj;
    }
    return status;
}

/* Number of OpenMP threads a call with nthreads <= 0 uses (1 without OpenMP). */
int orc_default_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
