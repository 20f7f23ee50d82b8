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
// one Newton-Raphson step for the reciprocal square root (y <- y (3 - r2 y^2)/2),
// which brings the relative error from ~1e-7 to ~1e-14.
// FP32 form (precision setting): positions relative to the target leaf centre
// in FP32, pairs in FP32 with Kahan-compensated accumulation; pairs closer than
// 1e-3 a (where the FP32 difference of coordinates loses the direction) are
// recomputed in FP64 from the FP64 positions.
#include <cmath>
#include <type_traits>

#include "rpy_internal.h"

namespace rpy {

constexpr double kPiD = 3.14159265358979323846;
constexpr int kP2PThreads = 256;

// Reciprocal square root: single-precision seed (relative error below 2^-21)
// and one Newton step, y (3 - r2 y^2) / 2 (error ~1e-14).  Valid while r2 is
// inside the float range; callers with r2 possibly outside use 1/sqrt.
__device__ __forceinline__ double rsqrt_newton(double r2) {
    double y = double(rsqrtf(float(r2)));
    return y * (1.5 - 0.5 * r2 * y * y);
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

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Source staging: the beads of all source boxes of a leaf's list are streamed
// through shared memory in chunks of blockDim, across box boundaries.  Every
// thread locates its bead of the chunk by walking the list from a uniform
// cursor (lists hold a few dozen boxes).
struct SrcCursor {
    int u, off;   // list position and offset inside that box
};

__device__ __forceinline__ int cursor_locate(SrcCursor c, int u1, int t, const int *uidx, const int *beg,
                                             const int *end) {
    int u = c.u, off = c.off;
    while (u < u1) {
        int C = uidx[u];
        int avail = end[C] - beg[C] - off;
        if (t < avail) return beg[C] + off + t;
        t -= avail;
        ++u;
        off = 0;
    }
    return -1;
}

__device__ __forceinline__ SrcCursor cursor_advance(SrcCursor c, int u1, int t, const int *uidx, const int *beg,
                                                    const int *end) {
    while (c.u < u1) {
        int C = uidx[c.u];
        int avail = end[C] - beg[C] - c.off;
        if (t < avail) {
            c.off += t;
            return c;
        }
        t -= avail;
        ++c.u;
        c.off = 0;
    }
    return c;
}

// Thread layout: a leaf of T beads uses R = min(T, blockDim) targets per pass and
// G = blockDim / R groups; group g takes every G-th bead of each staged chunk.
template <bool FP32>
__global__ void __launch_bounds__(kP2PThreads) k_p2p(const int *leaves, const int *beg, const int *end,
                                                     const int *bsys, const double *ctr, const int *uoff,
                                                     const int *uidx, const double *pos, const double *fs,
                                                     int64_t n, SysConst sc, int add_self, double *out) {
    using R_t = typename std::conditional<FP32, float, double>::type;
    __shared__ R_t sx[kP2PThreads], sy[kP2PThreads], sz[kP2PThreads];
    __shared__ R_t sfx[kP2PThreads], sfy[kP2PThreads], sfz[kP2PThreads];
    __shared__ int sj[kP2PThreads];
    __shared__ double red[3][kP2PThreads];
    int li = blockIdx.x;
    int b = leaves[li];
    int sys = bsys[b];
    double a = sc.a[sys], s = sc.s[sys];
    double co = s / (6.0 * kPiD * a);
    R_t a2x4 = R_t(4.0 * a * a), a2 = R_t(a * a), cf = R_t(s / (8.0 * kPiD));
    const float tiny2 = float(1e-6 * a * a), co32 = float(co), c9 = float(9.0 / (32.0 * a)), c3 = float(3.0 / (32.0 * a));
    const R_t k23 = R_t(2.0 * a * a / 3.0), k2 = R_t(2.0 * a * a);
    // far-branch pairs have r2 >= 4a^2; the float seed needs r2 inside the float range
    const bool safe_range = 4.0 * a * a > 1e-30 && 4.0 * a * a * 1e12 < 1e30;
    // FP32 works in coordinates relative to the target leaf centre
    double cx = FP32 ? ctr[3 * b] : 0.0, cy = FP32 ? ctr[3 * b + 1] : 0.0, cz = FP32 ? ctr[3 * b + 2] : 0.0;
    int u0 = uoff[li], u1 = uoff[li + 1];
    int nt = end[b] - beg[b];
    int Rn = nt < int(blockDim.x) ? nt : int(blockDim.x);
    int G = int(blockDim.x) / Rn;
    int tl = threadIdx.x % Rn, g = threadIdx.x / Rn;
    for (int i0 = beg[b]; i0 < end[b]; i0 += Rn) {
        int i = i0 + tl;
        bool act = i < end[b] && g < G;
        R_t xi = act ? R_t(pos[i] - cx) : R_t(0), yi = act ? R_t(pos[n + i] - cy) : R_t(0),
            zi = act ? R_t(pos[2 * n + i] - cz) : R_t(0);
        R_t acc[3] = {0, 0, 0}, cmp[3] = {0, 0, 0};
        double accd[3] = {0, 0, 0};
        SrcCursor cur{u0, 0};
        while (cur.u < u1) {
            __syncthreads();
            int j = cursor_locate(cur, u1, threadIdx.x, uidx, beg, end);
            sj[threadIdx.x] = j;
            if (j >= 0) {
                sx[threadIdx.x] = R_t(pos[j] - cx);
                sy[threadIdx.x] = R_t(pos[n + j] - cy);
                sz[threadIdx.x] = R_t(pos[2 * n + j] - cz);
                sfx[threadIdx.x] = R_t(fs[j]);
                sfy[threadIdx.x] = R_t(fs[n + j]);
                sfz[threadIdx.x] = R_t(fs[2 * n + j]);
            }
            cur = cursor_advance(cur, u1, int(blockDim.x), uidx, beg, end);
            __syncthreads();
            if (!act) continue;
            for (int jj = g; jj < int(blockDim.x); jj += G) {
                int jg = sj[jj];
                if (jg < 0) break;
                R_t dx = xi - sx[jj], dy = yi - sy[jj], dz = zi - sz[jj];
                R_t r2 = dx * dx + dy * dy + dz * dz;
                R_t fx = sfx[jj], fy = sfy[jj], fz = sfz[jj];
                if (r2 >= a2x4) {
                    // s/(8 pi r) [(1 + 2a^2/(3r^2)) F + (1 - 2a^2/r^2)(R.F)/r^2 R]
                    //   = t1 F + t2 R with A = cf/r, B = A/r^2
                    R_t ri;
                    if constexpr (FP32) ri = rsqrtf(r2);
                    else ri = safe_range ? rsqrt_newton(r2) : 1.0 / sqrt(r2);
                    R_t ri2 = ri * ri;
                    R_t A = cf * ri;
                    R_t B = A * ri2;
                    R_t RF = dx * fx + dy * fy + dz * fz;
                    R_t t1 = k23 * B + A;
                    R_t t2 = B * (R_t(1) - k2 * ri2) * RF;
                    if constexpr (FP32) {
                        kahan_add(acc[0], cmp[0], t1 * fx + t2 * dx);
                        kahan_add(acc[1], cmp[1], t1 * fy + t2 * dy);
                        kahan_add(acc[2], cmp[2], t1 * fz + t2 * dz);
                    } else {
                        acc[0] += t1 * fx + t2 * dx;
                        acc[1] += t1 * fy + t2 * dy;
                        acc[2] += t1 * fz + t2 * dz;
                    }
                } else if (jg != i) {
                    if constexpr (FP32) {
                        if (r2 > tiny2) {
                            // overlap branch in FP32: well conditioned away from r = 0
                            float r = sqrtf(r2);
                            float RF = dx * fx + dy * fy + dz * fz;
                            float t1 = co32 * (1.0f - c9 * r);
                            float t2 = co32 * c3 * RF / r;
                            kahan_add(acc[0], cmp[0], t1 * fx + t2 * dx);
                            kahan_add(acc[1], cmp[1], t1 * fy + t2 * dy);
                            kahan_add(acc[2], cmp[2], t1 * fz + t2 * dz);
                            continue;
                        }
                    }
                    // FP64 form, and beads within 1e-3 a of each other in the FP32 form
                    double ddx = pos[i] - pos[jg], ddy = pos[n + i] - pos[n + jg], ddz = pos[2 * n + i] - pos[2 * n + jg];
                    overlap_pair(ddx, ddy, ddz, ddx * ddx + ddy * ddy + ddz * ddz, fs[jg], fs[n + jg], fs[2 * n + jg], a,
                                 co, accd);
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
                for (int gg = 1; gg < G; ++gg) v[c] += red[c][threadIdx.x + gg * Rn];
            }
            double cs = add_self ? co : 0.0;
            out[3 * size_t(i)] = v[0] + cs * fs[i];
            out[3 * size_t(i) + 1] = v[1] + cs * fs[n + i];
            out[3 * size_t(i) + 2] = v[2] + cs * fs[2 * n + i];
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
        k_p2p<true><<<t.nleaf, kP2PThreads, 0, st>>>(t.leaves, t.b_begin, t.b_end, t.b_sys, t.b_center, off, idx,
                                                     t.pos, fs, t.n, sc, add_self, out);
        RPY_LAUNCHED(1);
    } else {
        k_p2p<false><<<t.nleaf, kP2PThreads, 0, st>>>(t.leaves, t.b_begin, t.b_end, t.b_sys, t.b_center, off, idx,
                                                      t.pos, fs, t.n, sc, add_self, out);
        RPY_LAUNCHED(1);
    }
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

}  // namespace rpy
