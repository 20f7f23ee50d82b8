/*
 * Plain, slow FP64 reference for the RPY matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library may include, link or call
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction,
 * so every operation below is one correctly rounded IEEE operation).
 *
 * Contents
 *   oracle_rpy_direct     u_i = sum_j D_ij F_j, Sec. 1 (RPY tensor, self term,
 *                          far branch Eq. "rpy-far", overlap branch).
 *   oracle_laplace_direct the Laplace potentials of Sec. 2 (L_k = sum q/|r_i-r_j|)
 *                          with gradient and Hessian, by direct summation.
 *   oracle_rpy_far_split  the far-field RPY velocity assembled from the four
 *                          Laplace potentials, Eq. (2.8), with the dipole term
 *                          -C2 grad L_C (see the reading below).
 *   oracle_morton_keys    bounding cube, 21-bit quantisation per axis and the
 *                          interleaved 63-bit Morton key of each bead (the tree
 *                          key; the paper only says the tree is adaptive with a
 *                          refinement limit, Sec. 4.2).
 *   oracle_stable_sort    stable merge sort of (key, index) pairs.
 *
 * Readings of the paper taken here (the paper is garbled or silent):
 *   - Overlap branch (r < 2a), Sec. 1: the printed prefactor kT/(6 pi eta r)
 *     and r(x)r/r^2 are dimensionally inconsistent and discontinuous at
 *     r = 2a.  The standard RPY overlap form is used:
 *       kT/(6 pi eta a) [ (1 - 9r/(32a)) I + (3/(32a)) r(x)r / r ].
 *     It is continuous with the far branch at r = 2a and tends to the self
 *     term as r -> 0.
 *   - r = 2a exactly takes the far branch (the paper's ">=").
 *   - Two distinct beads at the same point (r = 0) couple with the r -> 0
 *     limit of the overlap branch, kT/(6 pi eta a) I.
 *   - Eq. (2.8): the dipole term enters with a minus sign, -C2 grad L_C;
 *     the printed "+" contradicts the far branch of the tensor.
 *   - The boundary takes s = kT/eta; D is linear in s.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* One RPY block D_ij applied to F_j (i != j), added into u.  R = r_i - r_j. */
static void rpy_pair(const double R[3], const double F[3], double a, double s, double u[3])
{
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = sqrt(r2);
    double RF = R[0] * F[0] + R[1] * F[1] + R[2] * F[2];
    if (r >= 2.0 * a) {
        /* kT/(8 pi eta r) [ (I + RR/r^2) + 2a^2/(3r^2) (I - 3RR/r^2) ] F */
        double c = s / (8.0 * M_PI * r);
        double cf = c * (1.0 + 2.0 * a * a / (3.0 * r2));
        double cr = c * (1.0 - 2.0 * a * a / r2) * RF / r2;
        for (int k = 0; k < 3; ++k) u[k] += cf * F[k] + cr * R[k];
    } else if (r > 0.0) {
        /* kT/(6 pi eta a) [ (1 - 9r/(32a)) I + (3/(32a)) RR/r ] F */
        double c = s / (6.0 * M_PI * a);
        double cf = c * (1.0 - 9.0 * r / (32.0 * a));
        double cr = c * (3.0 / (32.0 * a)) * RF / r;
        for (int k = 0; k < 3; ++k) u[k] += cf * F[k] + cr * R[k];
    } else {
        double c = s / (6.0 * M_PI * a);
        for (int k = 0; k < 3; ++k) u[k] += c * F[k];
    }
}

/*
 * u[t] = D_{i i} F_i + sum_{j != i} D_ij F_j for each target i = targets[t].
 * pos, f: n x 3 row-major.  targets: nt indices (NULL means all beads).
 * Sources are summed in ascending j, so the result does not depend on the
 * thread count.
 */
void oracle_rpy_direct(const double *pos, const double *f, int64_t n, double a, double s,
                       const int64_t *targets, int64_t nt, double *u, int nthreads)
{
    if (targets == NULL) nt = n;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double acc[3] = {0.0, 0.0, 0.0};
        double self = s / (6.0 * M_PI * a);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) {
                for (int k = 0; k < 3; ++k) acc[k] += self * f[3 * j + k];
                continue;
            }
            double R[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                           pos[3 * i + 2] - pos[3 * j + 2]};
            rpy_pair(R, f + 3 * j, a, s, acc);
        }
        u[3 * t] = acc[0];
        u[3 * t + 1] = acc[1];
        u[3 * t + 2] = acc[2];
    }
}

/*
 * Laplace potentials of Sec. 2 by direct summation:
 *   phi_c(x)  = sum_j q[j*nq+c] / |x - y_j|
 * with gradient and Hessian with respect to x.  Sources that coincide with a
 * target are skipped.  Output per target t and charge set c:
 *   out[((t*nq)+c)*13 + 0]      potential
 *   out[...+1 .. +3]            gradient (x, y, z)
 *   out[...+4 .. +12]           Hessian, row-major 3x3
 */
void oracle_laplace_direct(const double *src, const double *q, int64_t ns, int nq,
                           const double *tgt, int64_t nt, double *out, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t t = 0; t < nt; ++t) {
        double *o = out + t * nq * 13;
        for (int c = 0; c < nq * 13; ++c) o[c] = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double R[3] = {tgt[3 * t] - src[3 * j], tgt[3 * t + 1] - src[3 * j + 1],
                           tgt[3 * t + 2] - src[3 * j + 2]};
            double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double g = 1.0 / r;               /* 1/r */
            double g3 = g / r2;               /* 1/r^3 */
            double g5 = g3 / r2;              /* 1/r^5 */
            for (int c = 0; c < nq; ++c) {
                double qj = q[j * nq + c];
                double *oc = o + c * 13;
                oc[0] += qj * g;
                for (int a = 0; a < 3; ++a) oc[1 + a] += -qj * R[a] * g3;      /* d/dx_a 1/r */
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)                                  /* d2/dx_a dx_b 1/r */
                        oc[4 + 3 * a + b] += qj * (3.0 * R[a] * R[b] * g5 - (a == b ? g3 : 0.0));
            }
        }
    }
}

/*
 * Far-field RPY velocity from the four Laplace potentials, Eq. (2.8):
 *   u = C1 [L1 L2 L3] - C1 (x grad L1 + y grad L2 + z grad L3) + C1 grad L4 - C2 grad L_C
 * with L1..L3 carrying F^1..F^3, L4 carrying F_j . r_j, L_C = dL1/dx + dL2/dy + dL3/dz,
 * C1 = s/(8 pi), C2 = s a^2/(12 pi).  Coordinates are taken relative to
 * `origin` (the identity holds for any common origin).  Every source j
 * contributes, except one that coincides with the target; the identity equals
 * the tensor only for pairs with r >= 2a.
 * dipole_sign = -1 is the correct reading; +1 reproduces the printed sign.
 */
void oracle_rpy_far_split(const double *pos_src, const double *f, int64_t ns,
                          const double *pos_tgt, int64_t nt, double a, double s,
                          const double origin[3], double dipole_sign, double *u, int nthreads)
{
    double *q = (double *)malloc(sizeof(double) * 4 * (ns > 0 ? ns : 1));
    double *ys = (double *)malloc(sizeof(double) * 3 * (ns > 0 ? ns : 1));
    double *xt = (double *)malloc(sizeof(double) * 3 * (nt > 0 ? nt : 1));
    double *lap = (double *)malloc(sizeof(double) * 4 * 13 * (nt > 0 ? nt : 1));
    for (int64_t j = 0; j < ns; ++j) {
        for (int k = 0; k < 3; ++k) ys[3 * j + k] = pos_src[3 * j + k] - origin[k];
        q[4 * j + 0] = f[3 * j + 0];
        q[4 * j + 1] = f[3 * j + 1];
        q[4 * j + 2] = f[3 * j + 2];
        q[4 * j + 3] = f[3 * j] * ys[3 * j] + f[3 * j + 1] * ys[3 * j + 1] + f[3 * j + 2] * ys[3 * j + 2];
    }
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) xt[3 * t + k] = pos_tgt[3 * t + k] - origin[k];
    oracle_laplace_direct(ys, q, ns, 4, xt, nt, lap, nthreads);
    double C1 = s / (8.0 * M_PI), C2 = s * a * a / (12.0 * M_PI);
    for (int64_t t = 0; t < nt; ++t) {
        const double *L = lap + t * 4 * 13;   /* L[c*13 + ...] */
        for (int d = 0; d < 3; ++d) {
            double v = C1 * L[d * 13 + 0];
            for (int k = 0; k < 3; ++k) v -= C1 * xt[3 * t + k] * L[k * 13 + 1 + d];
            v += C1 * L[3 * 13 + 1 + d];
            /* d/dx_d L_C = sum_k d2 L_k / dx_k dx_d */
            double dLC = 0.0;
            for (int k = 0; k < 3; ++k) dLC += L[k * 13 + 4 + 3 * k + d];
            v += dipole_sign * C2 * dLC;
            u[3 * t + d] = v;
        }
    }
    free(q);
    free(ys);
    free(xt);
    free(lap);
}

/*
 * Bounding cube and Morton keys.
 *   lo, hi  per-axis min / max;  side = max_k (hi_k - lo_k);
 *   centre_k = 0.5 (lo_k + hi_k);  origin_k = centre_k - 0.5 side;
 *   q_k = min(2^21 - 1, floor((x_k - origin_k) / side * 2^21)), 0 if side == 0
 *         (negative values from rounding clamp to 0);
 *   key  = bits of q interleaved from the most significant level down, each
 *          level contributing (z, y, x) in bit positions (3b+2, 3b+1, 3b).
 * cube[0..3] receives centre x, y, z and side.
 */
void oracle_morton_keys(const double *pos, int64_t n, uint64_t *keys, double *cube)
{
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = n ? pos[k] : 0.0; hi[k] = lo[k]; }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = pos[3 * i + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double side = 0.0;
    for (int k = 0; k < 3; ++k) { double e = hi[k] - lo[k]; if (e > side) side = e; }
    double centre[3], origin[3];
    for (int k = 0; k < 3; ++k) {
        centre[k] = 0.5 * (lo[k] + hi[k]);
        origin[k] = centre[k] - 0.5 * side;
    }
    cube[0] = centre[0]; cube[1] = centre[1]; cube[2] = centre[2]; cube[3] = side;
    const double scale = 2097152.0; /* 2^21 */
    for (int64_t i = 0; i < n; ++i) {
        uint64_t qk[3];
        for (int k = 0; k < 3; ++k) {
            if (side == 0.0) { qk[k] = 0; continue; }
            double t = (pos[3 * i + k] - origin[k]) / side;
            t = t * scale;
            double fl = floor(t);
            if (fl < 0.0) fl = 0.0;
            if (fl > scale - 1.0) fl = scale - 1.0;
            qk[k] = (uint64_t)fl;
        }
        uint64_t key = 0;
        for (int b = 20; b >= 0; --b) {
            key = (key << 3) | (((qk[2] >> b) & 1u) << 2) | (((qk[1] >> b) & 1u) << 1) | ((qk[0] >> b) & 1u);
        }
        keys[i] = key;
    }
}

/* Stable merge sort: perm receives indices 0..n-1 ordered by keys, ties in index order. */
void oracle_stable_sort(const uint64_t *keys, int64_t n, int64_t *perm)
{
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t a = lo, b = mid, o = lo;
            while (a < mid && b < hi) {
                if (keys[perm[b]] < keys[perm[a]]) tmp[o++] = perm[b++];
                else tmp[o++] = perm[a++];
            }
            while (a < mid) tmp[o++] = perm[a++];
            while (b < hi) tmp[o++] = perm[b++];
        }
        memcpy(perm, tmp, sizeof(int64_t) * n);
    }
    free(tmp);
}
