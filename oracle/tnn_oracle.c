/*
 * TEST INFRASTRUCTURE ONLY -- the CPU oracle for exact causal k-NN.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this file's library.  It shares no code, header, table or helper with
 * the CUDA path and must never be called from the product path.
 *
 * Everything here is the plain definition, written out in IEEE double with
 * no FMA contraction (compiled with -ffp-contract=off, no -ffast-math):
 *
 *   metric (Sec. 3.4, the scalable metric):
 *     d2(a, b) = ((sx*dx^2 + sy*dy^2) + sz*dz^2) + st*dt^2,
 *     d? = (double)b? - (double)a?;   sx = sy = sigma_xy in the paper, kept
 *     as two weights here (reading: a 4-vector of weights on squared
 *     differences).
 *   causal mask (Sec. 3.1 contexts hold only points at least t_w in the
 *     past; Eq. masked temporal part): point j is valid for a query at time
 *     t iff (double)t_j < (double)t - lag  (strict).
 *   k-NN: the k valid points with the smallest (d2, j) in lexicographic
 *     order; the ranking is exact, ties broken by the smaller index.  TNN is
 *     an exact method (Sec. 4.2, Table 3 caption), so this brute-force
 *     definition is the expected output of the whole search.
 *
 * Segment functions (Sec. 3.4, sets of K points approximated by the segment
 * from their first to their last point; Eq. projection on the segment;
 * Fig. 2) exist to check the index invariants; they play no part in the
 * k-NN oracle.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- metric */

double tnn_oracle_d2(const float *a, const float *b, const double *sigma)
{
    double dx = (double)b[0] - (double)a[0];
    double dy = (double)b[1] - (double)a[1];
    double dz = (double)b[2] - (double)a[2];
    double dt = (double)b[3] - (double)a[3];
    double s = sigma[0] * (dx * dx);
    s = s + sigma[1] * (dy * dy);
    s = s + sigma[2] * (dz * dz);
    s = s + sigma[3] * (dt * dt);
    return s;
}

/* ------------------------------------------------------------------ k-NN */

typedef struct {
    double d;
    int64_t j;
} cand_t;

static int cand_before(const cand_t *a, const cand_t *b)
{
    return a->d < b->d || (a->d == b->d && a->j < b->j);
}

/* k smallest valid points for one query, by plain sorted insertion. */
static void knn_one(const float *pts, int64_t n, const float *q,
                    const double *sigma, double lag, int k, cand_t *best,
                    int32_t *out_idx, float *out_d2, double *out_d64)
{
    const double tcut = (double)q[3] - lag;
    int cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        const float *p = pts + 4 * j;
        if (!((double)p[3] < tcut))
            continue;
        cand_t c;
        c.d = tnn_oracle_d2(q, p, sigma);
        c.j = j;
        if (cnt == k && !cand_before(&c, &best[k - 1]))
            continue;
        int pos = (cnt < k) ? cnt : k - 1;
        while (pos > 0 && cand_before(&c, &best[pos - 1])) {
            best[pos] = best[pos - 1];
            --pos;
        }
        best[pos] = c;
        if (cnt < k)
            ++cnt;
    }
    for (int r = 0; r < k; ++r) {
        if (r < cnt) {
            out_idx[r] = (int32_t)best[r].j;
            out_d2[r] = (float)best[r].d;
            if (out_d64)
                out_d64[r] = best[r].d;
        } else {
            out_idx[r] = -1;
            out_d2[r] = INFINITY;
            if (out_d64)
                out_d64[r] = INFINITY;
        }
    }
}

typedef struct {
    const float *pts;
    int64_t n;
    const float *qpts;
    const int64_t *qsel;
    int64_t m_begin, m_end;
    const double *sigma;
    double lag;
    int k;
    int32_t *out_idx;
    float *out_d2;
    double *out_d64;
} knn_job_t;

static void *knn_worker(void *arg)
{
    knn_job_t *jb = (knn_job_t *)arg;
    cand_t *best = (cand_t *)malloc(sizeof(cand_t) * (size_t)jb->k);
    if (!best)
        return (void *)1;
    for (int64_t i = jb->m_begin; i < jb->m_end; ++i) {
        int64_t qi = jb->qsel ? jb->qsel[i] : i;
        knn_one(jb->pts, jb->n, jb->qpts + 4 * qi, jb->sigma, jb->lag, jb->k,
                best, jb->out_idx + i * jb->k, jb->out_d2 + i * jb->k,
                jb->out_d64 ? jb->out_d64 + i * jb->k : NULL);
    }
    free(best);
    return NULL;
}

/*
 * Exact causal k-NN by brute force.
 *   pts      [n][4] float (x, y, z, t), the searched set
 *   qpts     [*][4] float, query rows (pass pts for self-query)
 *   qsel     optional row ids into qpts (m of them); NULL -> rows 0..m-1
 *   out_idx  [m][k] int32, -1 where fewer than k points are valid
 *   out_d2   [m][k] float = (float)d2 (round to nearest), +inf padding
 *   out_d64  optional [m][k] double, the FP64 d2
 * Returns 0 on success, -1 on a bad argument or thread failure.
 */
int tnn_oracle_knn(const float *pts, int64_t n, const float *qpts,
                   const int64_t *qsel, int64_t m, const double *sigma,
                   double lag, int32_t k, int32_t *out_idx, float *out_d2,
                   double *out_d64, int32_t nthreads)
{
    if (k < 1 || n < 0 || m < 0 || !pts || !qpts || !out_idx || !out_d2)
        return -1;
    if (nthreads < 1)
        nthreads = 1;
    if ((int64_t)nthreads > m)
        nthreads = (int32_t)(m > 0 ? m : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    knn_job_t *jobs = (knn_job_t *)malloc(sizeof(knn_job_t) * (size_t)nthreads);
    if (!th || !jobs) {
        free(th);
        free(jobs);
        return -1;
    }
    int rc = 0;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].pts = pts;
        jobs[t].n = n;
        jobs[t].qpts = qpts;
        jobs[t].qsel = qsel;
        jobs[t].m_begin = m * t / nthreads;
        jobs[t].m_end = m * (t + 1) / nthreads;
        jobs[t].sigma = sigma;
        jobs[t].lag = lag;
        jobs[t].k = k;
        jobs[t].out_idx = out_idx;
        jobs[t].out_d2 = out_d2;
        jobs[t].out_d64 = out_d64;
        if (pthread_create(&th[t], NULL, knn_worker, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) {
        void *ret = NULL;
        pthread_join(th[t], &ret);
        if (ret)
            rc = -1;
    }
    free(th);
    free(jobs);
    return rc;
}

/* ------------------------------------------------------------- segments */

/*
 * Distance in the sigma-scaled space from point p to the segment [a, b]
 * (Eq. projection on the segment, Fig. 2): the projection parameter
 * <ap, ab> / |ab|^2 is clamped to [0, 1]; a degenerate segment (a == b)
 * projects to a.  All coordinates are already scaled by sqrt(sigma).
 * Returns the squared distance.
 */
double tnn_oracle_point_segment_sq(const double *p, const double *a,
                                   const double *b)
{
    double ab[3], ap[3];
    for (int i = 0; i < 3; ++i) {
        ab[i] = b[i] - a[i];
        ap[i] = p[i] - a[i];
    }
    double ab2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    double lam = 0.0;
    if (ab2 > 0.0) {
        lam = (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / ab2;
        if (lam < 0.0)
            lam = 0.0;
        if (lam > 1.0)
            lam = 1.0;
    }
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
        double e = p[i] - (a[i] + lam * ab[i]);
        s += e * e;
    }
    return s;
}

static void scale3(const float *p, const double *sigma, double *out)
{
    out[0] = sqrt(sigma[0]) * (double)p[0];
    out[1] = sqrt(sigma[1]) * (double)p[1];
    out[2] = sqrt(sigma[2]) * (double)p[2];
}

/*
 * Segment table in build order (Sec. 3.4: each time-sorted trajectory is cut
 * into consecutive sets of K points; reading: the last set of a trajectory
 * keeps its n mod K points instead of padding with copies).
 *   traj_off [T+1]; returns the number of segments, or -1 if out_cap is too
 *   small.  Per segment s: first[s], count[s], A[s][3], B[s][3] (scaled by
 *   sqrt(sigma)), tA[s], tB[s], radius[s] = max over members of the
 *   Euclidean distance (scaled space) to the segment [A, B].
 */
int64_t tnn_oracle_segments(const float *pts, const int64_t *traj_off,
                            int64_t n_traj, const double *sigma, int32_t K,
                            int64_t out_cap, int64_t *first, int32_t *count,
                            double *A, double *B, double *tA, double *tB,
                            double *radius)
{
    if (K < 1)
        return -1;
    int64_t s = 0;
    for (int64_t tr = 0; tr < n_traj; ++tr) {
        for (int64_t f = traj_off[tr]; f < traj_off[tr + 1]; f += K) {
            int64_t e = f + K;
            if (e > traj_off[tr + 1])
                e = traj_off[tr + 1];
            if (s >= out_cap)
                return -1;
            first[s] = f;
            count[s] = (int32_t)(e - f);
            scale3(pts + 4 * f, sigma, A + 3 * s);
            scale3(pts + 4 * (e - 1), sigma, B + 3 * s);
            tA[s] = (double)pts[4 * f + 3];
            tB[s] = (double)pts[4 * (e - 1) + 3];
            double r2 = 0.0;
            for (int64_t j = f; j < e; ++j) {
                double pj[3];
                scale3(pts + 4 * j, sigma, pj);
                double d = tnn_oracle_point_segment_sq(pj, A + 3 * s, B + 3 * s);
                if (d > r2)
                    r2 = d;
            }
            radius[s] = sqrt(r2);
            ++s;
        }
    }
    return s;
}

/*
 * Lower bound on d2(q, j) over the valid points j of one segment
 * (the cylinder reading of the exclusion criterion of Sec. 3.4):
 *   +inf                                   if tA >= t_q - lag (Eq. masked
 *                                          temporal part: nothing valid);
 *   max(0, dist(q', [A, B]) - r)^2 + st * max(t_q - tB, lag)^2 otherwise.
 * Every valid point lies within r of the segment (triangle inequality) and
 * has tB >= t_j, t_q - t_j > lag.  q is a raw float query (x, y, z, t).
 */
double tnn_oracle_cylinder_lb(const float *q, const double *sigma, double lag,
                              const double *A, const double *B, double tA,
                              double tB, double r)
{
    double tq = (double)q[3];
    if (!(tA < tq - lag))
        return INFINITY;
    double qs[3];
    scale3(q, sigma, qs);
    double a = sqrt(tnn_oracle_point_segment_sq(qs, A, B)) - r;
    if (a < 0.0)
        a = 0.0;
    double dt = tq - tB;
    if (dt < lag)
        dt = lag;
    return a * a + sigma[3] * dt * dt;
}

/*
 * Algorithm 1 exactly as printed (mask, clamp, squared distance to the
 * projected point, temporal term max(t_B - t, 0)^2, then subtract
 * E * max(sigma_xy, sigma_z) and clamp at 0), with E the squared
 * approximation error E_app in Euclidean units.  Kept only so that a test
 * can show where it stops being a lower bound (reading of the exclusion
 * criterion); the search never uses it.
 */
double tnn_oracle_paper_alg1(const float *q, const double *sigma, double lag,
                             const double *A_raw, const double *B_raw,
                             double tA, double tB, double E_euclid_sq)
{
    double tq = (double)q[3];
    if (tA > tq - lag)
        return INFINITY;
    double ab[3], ap[3];
    for (int i = 0; i < 3; ++i) {
        ab[i] = B_raw[i] - A_raw[i];
        ap[i] = (double)q[i] - A_raw[i];
    }
    double ab2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    double lam = 0.0;
    if (ab2 > 0.0)
        lam = (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / ab2;
    if (lam < 0.0)
        lam = 0.0;
    if (lam > 1.0)
        lam = 1.0;
    double D = 0.0;
    for (int i = 0; i < 3; ++i) {
        double e = (A_raw[i] + lam * ab[i]) - (double)q[i];
        D += sigma[i] * e * e;
    }
    double tt = tB - tq;
    if (tt < 0.0)
        tt = 0.0;
    D += sigma[3] * tt * tt;
    double smax = sigma[0] > sigma[2] ? sigma[0] : sigma[2];
    if (sigma[1] > smax)
        smax = sigma[1];
    D -= E_euclid_sq * smax;
    return D > 0.0 ? D : 0.0;
}
