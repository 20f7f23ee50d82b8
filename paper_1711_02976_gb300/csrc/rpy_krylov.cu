// Consumers of repeated matvecs on a resident tree (Sec. 1: Brownian dynamics
// needs D F for the drift and a vector with covariance 2 dt D for the noise):
//
//   rpy_lanczos_sqrt  y ~ D^{1/2} z by the Lanczos process on D: with the
//                     orthonormal Krylov basis V_m of (D, z) and the tridiagonal
//                     T_m = V_m^T D V_m, y_m = |z| V_m T_m^{1/2} e_1.  The step
//                     stops when the relative change of y between successive m
//                     falls below the tolerance (the change is computed from the
//                     small coefficient vectors, V_m being orthonormal).
//   rpy_bd_step       one Ermak-McCammon step without the divergence term (the
//                     divergence of the RPY tensor vanishes):
//                     r <- r + (dt/kT) D F + sqrt(2 dt) D^{1/2} xi, then the tree is
//                     rebuilt for the new positions.
//
// Vectors live on the device (3N doubles, caller order); the Lanczos
// coefficients and the square root of the small tridiagonal matrix (cyclic
// Jacobi rotations, m x m) are host work.  Dot products are deterministic
// (fixed grid, fixed reduction order).
#include <algorithm>
#include <cmath>
#include <vector>

#include "rpy_internal.h"

namespace rpy {

constexpr int kKThreads = 256;
constexpr int kKBlocks = 304;   // two per SM of a GB300

__global__ void k_dot_part(const double *x, const double *y, int64_t n, double *part) {
    __shared__ double red[kKThreads];
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        acc = fma(x[i], y[i], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kKThreads / 2; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// y = a x + b y
__global__ void k_axpby(double a, const double *x, double b, double *y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = fma(a, x[i], b * y[i]);
}

// y = sum_k c[k] V[k]
__global__ void k_lincomb(const double *V, int m, const double *c, int64_t n, double *y) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(c[k], V[size_t(k) * n + i], acc);
        y[i] = acc;
    }
}

// r <- r + (dt / kT_s) u + sqrt(2 dt) y for every bead of system s
__global__ void k_bd_update(double *pos, const double *u, const double *y, const int64_t *off, int nsys,
                            const double *dt_over_kT, double sq2dt, int64_t n) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsys;   // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    const double c = dt_over_kT[lo];
    for (int d = 0; d < 3; ++d) pos[3 * i + d] += fma(c, u[3 * i + d], sq2dt * y[3 * i + d]);
}

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

int dot(const double *x, const double *y, int64_t n, double *part_dev, double *out, cudaStream_t st) {
    k_dot_part<<<kKBlocks, kKThreads, 0, st>>>(x, y, n, part_dev);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    double part[kKBlocks];
    RPY_CHECK(cudaMemcpyAsync(part, part_dev, sizeof(part), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : part) s += v;
    *out = s;
    return RPY_OK;
}

int axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t st) {
    k_axpby<<<kKBlocks, kKThreads, 0, st>>>(a, x, b, y, n);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

// c = T^{1/2} e_1 for the symmetric tridiagonal T (diagonal al[0..m), off-diagonal
// be[0..m-1)), by cyclic Jacobi rotations on the dense m x m matrix: A = Q L Q^T,
// T^{1/2} e_1 = Q sqrt(L) Q^T e_1.  Eigenvalues below zero (rounding of a nearly
// singular T) are taken as zero.
void tridiag_sqrt_e1(const std::vector<double> &al, const std::vector<double> &be, int m, std::vector<double> &c) {
    std::vector<double> A(size_t(m) * m, 0.0), Q(size_t(m) * m, 0.0);
    for (int i = 0; i < m; ++i) {
        A[size_t(i) * m + i] = al[i];
        Q[size_t(i) * m + i] = 1.0;
        if (i + 1 < m) A[size_t(i) * m + i + 1] = A[size_t(i + 1) * m + i] = be[i];
    }
    double scale = 0.0;
    for (double v : A) scale = std::max(scale, std::fabs(v));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off = std::max(off, std::fabs(A[size_t(p) * m + q]));
        if (off <= 1e-17 * scale) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[size_t(p) * m + q];
                if (apq == 0.0) continue;
                // rotation zeroing A[p][q]: t = tan(theta), theta from cot(2 theta) = (a_qq - a_pp) / (2 a_pq)
                const double th = (A[size_t(q) * m + q] - A[size_t(p) * m + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < m; ++k) {   // columns p, q of A
                    const double akp = A[size_t(k) * m + p], akq = A[size_t(k) * m + q];
                    A[size_t(k) * m + p] = cs * akp - sn * akq;
                    A[size_t(k) * m + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < m; ++k) {   // rows p, q
                    const double apk = A[size_t(p) * m + k], aqk = A[size_t(q) * m + k];
                    A[size_t(p) * m + k] = cs * apk - sn * aqk;
                    A[size_t(q) * m + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < m; ++k) {   // eigenvectors: columns of Q
                    const double qkp = Q[size_t(k) * m + p], qkq = Q[size_t(k) * m + q];
                    Q[size_t(k) * m + p] = cs * qkp - sn * qkq;
                    Q[size_t(k) * m + q] = sn * qkp + cs * qkq;
                }
            }
    }
    c.assign(m, 0.0);
    for (int k = 0; k < m; ++k) {
        const double lam = std::max(0.0, A[size_t(k) * m + k]);
        const double w = std::sqrt(lam) * Q[k];   // sqrt(lambda_k) (Q^T e_1)_k
        for (int i = 0; i < m; ++i) c[i] += w * Q[size_t(i) * m + k];
    }
}

// Lanczos on the tree's D; y_dev receives |z| V_m T_m^{1/2} e_1.
int lanczos_sqrt(rpy_tree h, Tree &t, const double *z, const double *s_host, int m_max, double tol, double *y,
                 int *iters, double *est, cudaStream_t st) {
    const int64_t n3 = 3 * t.n;
    DevBuf bv, bw, bp, bc;
    RPY_CHECK(cudaMalloc(&bv.p, sizeof(double) * size_t(m_max + 1) * n3));
    RPY_CHECK(cudaMalloc(&bw.p, sizeof(double) * n3));
    RPY_CHECK(cudaMalloc(&bp.p, sizeof(double) * kKBlocks));
    RPY_CHECK(cudaMalloc(&bc.p, sizeof(double) * (m_max + 1)));
    double *V = static_cast<double *>(bv.p), *w = static_cast<double *>(bw.p), *part = static_cast<double *>(bp.p);
    double *cdev = static_cast<double *>(bc.p);
    double zz = 0.0;
    RPY_TRY(dot(z, z, n3, part, &zz, st));
    if (iters) *iters = 0;
    if (est) *est = 0.0;
    if (!std::isfinite(zz)) return RPY_ERR_NONFINITE;
    if (zz == 0.0) {
        RPY_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * n3, st));
        RPY_CHECK(cudaStreamSynchronize(st));
        return RPY_OK;
    }
    const double nz = std::sqrt(zz);
    RPY_CHECK(cudaMemsetAsync(V, 0, sizeof(double) * n3, st));
    RPY_TRY(axpby(1.0 / nz, z, 0.0, V, n3, st));
    std::vector<double> al, be, c, cprev;
    double change = INFINITY;
    int m = 0;
    for (int j = 0; j < m_max; ++j) {
        const double *vj = V + size_t(j) * n3;
        RPY_TRY(rpy_forest_matvec(h, vj, s_host, w, st));
        if (j > 0) RPY_TRY(axpby(-be[j - 1], V + size_t(j - 1) * n3, 1.0, w, n3, st));
        double a = 0.0;
        RPY_TRY(dot(w, vj, n3, part, &a, st));
        RPY_TRY(axpby(-a, vj, 1.0, w, n3, st));
        double bb = 0.0;
        RPY_TRY(dot(w, w, n3, part, &bb, st));
        if (!std::isfinite(a) || !std::isfinite(bb)) return RPY_ERR_NONFINITE;
        al.push_back(a);
        m = j + 1;
        tridiag_sqrt_e1(al, be, m, c);
        for (double &v : c) v *= nz;
        if (j > 0) {
            double dn = 0.0, cn = 0.0;
            for (int i = 0; i < m; ++i) {
                const double d = c[i] - (i < m - 1 ? cprev[i] : 0.0);
                dn += d * d;
                cn += c[i] * c[i];
            }
            change = std::sqrt(dn / cn);
        }
        cprev = c;
        const double b = std::sqrt(bb);
        // converged, or the Krylov space is exhausted (invariant subspace)
        if ((j > 0 && change <= tol) || b <= 1e-14 * std::sqrt(std::fabs(a) * std::fabs(a) + bb) || j + 1 == m_max)
            break;
        be.push_back(b);
        double *vn = V + size_t(j + 1) * n3;
        RPY_CHECK(cudaMemsetAsync(vn, 0, sizeof(double) * n3, st));
        RPY_TRY(axpby(1.0 / b, w, 0.0, vn, n3, st));
    }
    RPY_CHECK(cudaMemcpyAsync(cdev, c.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    k_lincomb<<<kKBlocks, kKThreads, 0, st>>>(V, m, cdev, n3, y);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_CHECK(cudaStreamSynchronize(st));
    if (iters) *iters = m;
    if (est) *est = change;
    return RPY_OK;
}

}  // namespace
}  // namespace rpy

using namespace rpy;

extern "C" int rpy_lanczos_sqrt(rpy_tree h, const double *z_dev, const double *kT_over_eta_host, int m_max, double tol,
                                double *y_dev, int *iters, double *rel_change, void *stream) {
    Tree *t = tree_of(h);
    if (!t || !z_dev || !y_dev || !kT_over_eta_host || m_max < 1 || m_max > 1000 || !(tol >= 0.0)) return RPY_ERR_INVALID;
    for (int k = 0; k < t->nsys; ++k)
        if (!(kT_over_eta_host[k] >= 0.0) || !std::isfinite(kT_over_eta_host[k])) return RPY_ERR_INVALID;
    DeviceGuard g(t->device);
    return lanczos_sqrt(h, *t, z_dev, kT_over_eta_host, m_max, tol, y_dev, iters, rel_change,
                        static_cast<cudaStream_t>(stream));
}

extern "C" int rpy_bd_step(rpy_tree h, double *pos_dev, const double *f_dev, const double *xi_dev,
                           const double *kT_host, const double *eta_host, double dt, int m_max, double tol,
                           double *disp_dev, int *iters, void *stream) {
    Tree *t = tree_of(h);
    if (!t || !pos_dev || !f_dev || !xi_dev || !kT_host || !eta_host || !(dt >= 0.0) || !std::isfinite(dt) ||
        m_max < 1 || m_max > 1000 || !(tol >= 0.0))
        return RPY_ERR_INVALID;
    std::vector<double> s(t->nsys), c(t->nsys);
    for (int k = 0; k < t->nsys; ++k) {
        if (!(kT_host[k] > 0.0) || !(eta_host[k] > 0.0) || !std::isfinite(kT_host[k]) || !std::isfinite(eta_host[k]))
            return RPY_ERR_INVALID;
        s[k] = kT_host[k] / eta_host[k];
        c[k] = dt / kT_host[k];
    }
    DeviceGuard g(t->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = t->n, n3 = 3 * n;
    DevBuf bu, by, bc;
    RPY_CHECK(cudaMalloc(&bu.p, sizeof(double) * n3));
    RPY_CHECK(cudaMalloc(&by.p, sizeof(double) * n3));
    RPY_CHECK(cudaMalloc(&bc.p, sizeof(double) * t->nsys));
    double *u = static_cast<double *>(bu.p), *y = static_cast<double *>(by.p), *cd = static_cast<double *>(bc.p);
    RPY_TRY(rpy_forest_matvec(h, f_dev, s.data(), u, stream));
    RPY_TRY(lanczos_sqrt(h, *t, xi_dev, s.data(), m_max, tol, y, iters, nullptr, st));
    RPY_CHECK(cudaMemcpyAsync(cd, c.data(), sizeof(double) * t->nsys, cudaMemcpyHostToDevice, st));
    if (disp_dev) {
        RPY_CHECK(cudaMemsetAsync(disp_dev, 0, sizeof(double) * n3, st));
        k_bd_update<<<unsigned((n + 255) / 256), 256, 0, st>>>(disp_dev, u, y, t->sys_off, t->nsys, cd,
                                                                std::sqrt(2.0 * dt), n);
        RPY_LAUNCHED(1);
    }
    k_bd_update<<<unsigned((n + 255) / 256), 256, 0, st>>>(pos_dev, u, y, t->sys_off, t->nsys, cd, std::sqrt(2.0 * dt),
                                                            n);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    return rpy_tree_update_positions(h, pos_dev, stream);
}
