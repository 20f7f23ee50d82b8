// Near field: direct RPY tensor (Sec. 1) over the U list of every leaf, the
// self term, and the final combine / unpermute of the matvec.
//
// One CTA per target leaf; its beads are the threads.  Source leaves of the U
// list are staged through shared memory in chunks of blockDim beads
// (coalesced SoA loads), and every thread sums its own target.
//
// Pair blocks (R = r_i - r_j, s = kT/eta):
//   r >= 2a : s/(8 pi r) [ (1 + 2a^2/(3r^2)) F + (1 - 2a^2/r^2) (R.F)/r^2 R ]
//   0<r<2a  : s/(6 pi a) [ (1 - 9r/(32a)) F + (3/(32a)) (R.F)/r R ]   (standard overlap form)
//   r = 0   : s/(6 pi a) F                                           (r -> 0 limit)
// The self term s/(6 pi a) F_i is added once.
//
// FP64 form: every operation in FP64; 1/r from a single-precision seed and
// two Newton-Raphson steps for the reciprocal square root (y <- y (3 - r2 y^2)/2),
// which restores full double precision.
// FP32 form (precision setting): positions relative to the target leaf centre
// in FP32, far-branch pairs in FP32 with Kahan-compensated accumulation;
// overlap pairs (r < 2a) recomputed in FP64 from the FP64 positions.
#include <cmath>

#include "rpy_internal.h"

namespace rpy {

constexpr double kPiD = 3.14159265358979323846;
constexpr int kP2PThreads = 128;

__device__ __forceinline__ double rsqrt_newton(double r2) {
    if (r2 < 1e-30 || r2 > 1e30) return 1.0 / sqrt(r2);
    double y = double(rsqrtf(float(r2)));
    y = y * (1.5 - 0.5 * r2 * y * y);
    y = y * (1.5 - 0.5 * r2 * y * y);
    return y;
}

__device__ __forceinline__ void overlap_pair(double dx, double dy, double dz, double r2, double fx, double fy, double fz,
                                             double a, double co, double *acc) {
    if (r2 > 0.0) {
        double r = sqrt(r2);
        double RF = dx * fx + dy * fy + dz * fz;
        double t1 = co * (1.0 - 9.0 * r / (32.0 * a));
        double t2 = co * (3.0 / (32.0 * a)) * RF / r;
        acc[0] += t1 * fx + t2 * dx;
        acc[1] += t1 * fy + t2 * dy;
        acc[2] += t1 * fz + t2 * dz;
    } else {
        acc[0] += co * fx;
        acc[1] += co * fy;
        acc[2] += co * fz;
    }
}

__global__ void __launch_bounds__(kP2PThreads) k_p2p64(const int *leaves, const int *beg, const int *end,
                                                        const int *bsys, const int *uoff, const int *uidx,
                                                        const double *pos, const double *fs, int64_t n, SysConst sc,
                                                        int add_self, double *unear) {
    __shared__ double sx[kP2PThreads], sy[kP2PThreads], sz[kP2PThreads];
    __shared__ double sfx[kP2PThreads], sfy[kP2PThreads], sfz[kP2PThreads];
    __shared__ double red[3][kP2PThreads];
    int li = blockIdx.x;
    int b = leaves[li];
    int sys = bsys[b];
    double a = sc.a[sys], s = sc.s[sys];
    double a2x4 = 4.0 * a * a, a2 = a * a;
    double cf = s / (8.0 * kPiD), co = s / (6.0 * kPiD * a);
    int u0 = uoff[li], u1 = uoff[li + 1];
    // R targets per pass (a multiple of the warp size), G groups splitting the sources
    int nt = end[b] - beg[b];
    int R = nt >= int(blockDim.x) ? int(blockDim.x) : ((nt + 31) & ~31);
    int G = int(blockDim.x) / R;
    int tl = threadIdx.x % R, g = threadIdx.x / R;
    for (int i0 = beg[b]; i0 < end[b]; i0 += R) {
        int i = i0 + tl;
        bool act = i < end[b] && g < G;
        double xi = act ? pos[i] : 0, yi = act ? pos[n + i] : 0, zi = act ? pos[2 * n + i] : 0;
        double acc[3] = {0, 0, 0};
        for (int u = u0; u < u1; ++u) {
            int C = uidx[u];
            for (int j0 = beg[C]; j0 < end[C]; j0 += blockDim.x) {
                int cnt = min(int(blockDim.x), end[C] - j0);
                __syncthreads();
                if (threadIdx.x < cnt) {
                    int j = j0 + threadIdx.x;
                    sx[threadIdx.x] = pos[j];
                    sy[threadIdx.x] = pos[n + j];
                    sz[threadIdx.x] = pos[2 * n + j];
                    sfx[threadIdx.x] = fs[j];
                    sfy[threadIdx.x] = fs[n + j];
                    sfz[threadIdx.x] = fs[2 * n + j];
                }
                __syncthreads();
                if (!act) continue;
                for (int jj = g; jj < cnt; jj += G) {
                    double dx = xi - sx[jj], dy = yi - sy[jj], dz = zi - sz[jj];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    double fx = sfx[jj], fy = sfy[jj], fz = sfz[jj];
                    if (r2 >= a2x4) {
                        double ri = rsqrt_newton(r2);
                        double ri2 = ri * ri;
                        double c = cf * ri;
                        double q = a2 * ri2;
                        double RF = dx * fx + dy * fy + dz * fz;
                        double t1 = c * (1.0 + (2.0 / 3.0) * q);
                        double t2 = c * (1.0 - 2.0 * q) * RF * ri2;
                        acc[0] += t1 * fx + t2 * dx;
                        acc[1] += t1 * fy + t2 * dy;
                        acc[2] += t1 * fz + t2 * dz;
                    } else if (j0 + jj != i) {
                        overlap_pair(dx, dy, dz, r2, fx, fy, fz, a, co, acc);
                    }
                }
            }
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
        __syncthreads();
        if (act && g == 0) {
            for (int gg = 1; gg < G; ++gg)
                for (int c = 0; c < 3; ++c) acc[c] += red[c][threadIdx.x + gg * R];
            double cs = add_self ? co : 0.0;
            unear[3 * size_t(i)] = acc[0] + cs * fs[i];
            unear[3 * size_t(i) + 1] = acc[1] + cs * fs[n + i];
            unear[3 * size_t(i) + 2] = acc[2] + cs * fs[2 * n + i];
        }
    }
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

__global__ void __launch_bounds__(kP2PThreads) k_p2p32(const int *leaves, const int *beg, const int *end,
                                                        const int *bsys, const double *ctr, const int *uoff,
                                                        const int *uidx, const double *pos, const double *fs,
                                                        int64_t n, SysConst sc, int add_self, double *unear) {
    __shared__ float sx[kP2PThreads], sy[kP2PThreads], sz[kP2PThreads];
    __shared__ float sfx[kP2PThreads], sfy[kP2PThreads], sfz[kP2PThreads];
    __shared__ double red[3][kP2PThreads];
    int li = blockIdx.x;
    int b = leaves[li];
    int sys = bsys[b];
    double a = sc.a[sys], s = sc.s[sys];
    float a2x4 = float(4.0 * a * a), a2 = float(a * a);
    float cf = float(s / (8.0 * kPiD));
    double co = s / (6.0 * kPiD * a);
    double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2];
    int u0 = uoff[li], u1 = uoff[li + 1];
    int nt = end[b] - beg[b];
    int R = nt >= int(blockDim.x) ? int(blockDim.x) : ((nt + 31) & ~31);
    int G = int(blockDim.x) / R;
    int tl = threadIdx.x % R, g = threadIdx.x / R;
    for (int i0 = beg[b]; i0 < end[b]; i0 += R) {
        int i = i0 + tl;
        bool act = i < end[b] && g < G;
        float xi = act ? float(pos[i] - cx) : 0.f, yi = act ? float(pos[n + i] - cy) : 0.f,
              zi = act ? float(pos[2 * n + i] - cz) : 0.f;
        float acc[3] = {0, 0, 0}, cmp[3] = {0, 0, 0};
        double accd[3] = {0, 0, 0};
        for (int u = u0; u < u1; ++u) {
            int C = uidx[u];
            for (int j0 = beg[C]; j0 < end[C]; j0 += blockDim.x) {
                int cnt = min(int(blockDim.x), end[C] - j0);
                __syncthreads();
                if (threadIdx.x < cnt) {
                    int j = j0 + threadIdx.x;
                    sx[threadIdx.x] = float(pos[j] - cx);
                    sy[threadIdx.x] = float(pos[n + j] - cy);
                    sz[threadIdx.x] = float(pos[2 * n + j] - cz);
                    sfx[threadIdx.x] = float(fs[j]);
                    sfy[threadIdx.x] = float(fs[n + j]);
                    sfz[threadIdx.x] = float(fs[2 * n + j]);
                }
                __syncthreads();
                if (!act) continue;
                for (int jj = g; jj < cnt; jj += G) {
                    float dx = xi - sx[jj], dy = yi - sy[jj], dz = zi - sz[jj];
                    float r2 = dx * dx + dy * dy + dz * dz;
                    float fx = sfx[jj], fy = sfy[jj], fz = sfz[jj];
                    if (r2 >= a2x4) {
                        float ri = rsqrtf(r2);
                        float ri2 = ri * ri;
                        float c = cf * ri;
                        float q = a2 * ri2;
                        float RF = dx * fx + dy * fy + dz * fz;
                        float t1 = c * (1.0f + (2.0f / 3.0f) * q);
                        float t2 = c * (1.0f - 2.0f * q) * RF * ri2;
                        kahan_add(acc[0], cmp[0], t1 * fx + t2 * dx);
                        kahan_add(acc[1], cmp[1], t1 * fy + t2 * dy);
                        kahan_add(acc[2], cmp[2], t1 * fz + t2 * dz);
                    } else if (j0 + jj != i) {
                        int j = j0 + jj;
                        double ddx = pos[i] - pos[j], ddy = pos[n + i] - pos[n + j], ddz = pos[2 * n + i] - pos[2 * n + j];
                        overlap_pair(ddx, ddy, ddz, ddx * ddx + ddy * ddy + ddz * ddz, fs[j], fs[n + j], fs[2 * n + j],
                                     a, co, accd);
                    }
                }
            }
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = (double(acc[c]) - double(cmp[c])) + accd[c];
        __syncthreads();
        if (act && g == 0) {
            double v[3];
            for (int c = 0; c < 3; ++c) {
                v[c] = red[c][threadIdx.x];
                for (int gg = 1; gg < G; ++gg) v[c] += red[c][threadIdx.x + gg * R];
            }
            double cs = add_self ? co : 0.0;
            unear[3 * size_t(i)] = v[0] + cs * fs[i];
            unear[3 * size_t(i) + 1] = v[1] + cs * fs[n + i];
            unear[3 * size_t(i) + 2] = v[2] + cs * fs[2 * n + i];
        }
    }
}

// U lists (near field, self term added) or the direct substitutes of small
// W / X interactions (no self term).
int run_p2p(Tree &t, const double *fs, double *out, const SysConst &sc, cudaStream_t st, bool direct_list) {
    const int *off = direct_list ? t.d_off : t.u_off;
    const int *idx = direct_list ? t.d_idx : t.u_idx;
    int add_self = direct_list ? 0 : 1;
    if (t.params.precision == RPY_FP32) {
        k_p2p32<<<t.nleaf, kP2PThreads, 0, st>>>(t.leaves, t.b_begin, t.b_end, t.b_sys, t.b_center, off, idx, t.pos,
                                                 fs, t.n, sc, add_self, out);
        RPY_LAUNCHED(1);
    } else {
        k_p2p64<<<t.nleaf, kP2PThreads, 0, st>>>(t.leaves, t.b_begin, t.b_end, t.b_sys, off, idx, t.pos, fs, t.n, sc,
                                                 add_self, out);
        RPY_LAUNCHED(1);
    }
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

}  // namespace rpy
