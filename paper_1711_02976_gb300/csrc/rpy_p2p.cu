// Near field: direct RPY tensor (Sec. 1) over the U list of every leaf, the
// self term, and the final combine / unpermute of the matvec.
//
// One CTA per work item: up to 256 target beads of one leaf (large leaves are
// split into several items, launched in decreasing order of cost).  The beads of
// the leaf's source boxes are staged through shared memory in chunks (coalesced
// SoA loads) and every thread sums its own targets.
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
// FP32 form (precision setting, k_p2p32): positions relative to the target
// leaf centre in FP32; every thread carries two targets as the two lanes of
// packed FP32x2 operations and takes two staged sources per iteration; an
// iteration whose pairs are all far (across the warp) evaluates the far branch
// alone on the packed pairs, any other evaluates both branches per target with
// selects; accumulation is Kahan-compensated across blocks of kP32Block sources;
// pairs closer than 1e-3 a (where the FP32 difference of coordinates loses the
// direction) are recomputed in FP64 from the FP64 positions.
#include <cmath>

#include <mutex>
#include <set>

#include "rpy_internal.h"

namespace rpy {

constexpr double kPiD = 3.14159265358979323846;
constexpr int kP2PThreads = 256;

// Reciprocal square root for r2 > 0: an FP32 seed taken from the bit pattern
// of r2 (exponent rebased from 1023 to 127, mantissa truncated to 23 bits, by
// integer operations only), rsqrtf of it, and one Newton step in FP64,
//   e = 1 - r2 y0^2,  y = y0 + (y0/2) e      (relative error ~1.5 d^2 for a seed error d),
// with y0/2 formed by decrementing the exponent.  Returns false when r2 lies
// outside the normal FP32 range; the caller then takes 1/sqrt(r2).
__device__ __forceinline__ bool rsqrt_seeded(double r2, double &ri) {
    const unsigned hi = unsigned(__double2hiint(r2)), lo = unsigned(__double2loint(r2));
    const unsigned he = hi - (896u << 20);
    if (he - (1u << 20) >= (254u << 20)) return false;   // FP32 exponent outside [1, 254]
    const float y0f = rsqrtf(__uint_as_float(__funnelshift_l(lo, he, 3)));
    const unsigned yb = __float_as_uint(y0f);
    const double y0 = __hiloint2double(int((yb >> 3) + (896u << 20)), int(yb << 29));
    const double y0h = __hiloint2double(int((yb >> 3) + (895u << 20)), int(yb << 29));
    const double e = fma(-r2 * y0, y0, 1.0);
    ri = fma(y0h, e, y0);
    return true;
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
// Far pairs accumulate in units of s/(8 pi) (applied once per target) with
// explicit FMAs: 24 FP64 operations per pair and no conversions.
__global__ void __launch_bounds__(kP2PThreads) k_p2p(const int2 *items, const int *leaves, const int *beg,
                                                     const int *end, const int *bsys, const int *uoff,
                                                     const int *uidx, const double *pos, const double *fs, int64_t n,
                                                     SysConst sc, int add_self, double *out) {
    __shared__ double sx[kP2PThreads], sy[kP2PThreads], sz[kP2PThreads];
    __shared__ double sfx[kP2PThreads], sfy[kP2PThreads], sfz[kP2PThreads];
    __shared__ int sj[kP2PThreads];
    __shared__ double red[3][kP2PThreads];
    const int2 item = items[blockIdx.x];
    const int li = item.x, b = leaves[li], sys = bsys[b];
    const int tb = item.y, te = min(end[b], item.y + kItemTargets);
    const PairConst &pc = sc.pc[sys];
    const double a = pc.a, co = pc.co, cf = pc.cf, k23 = pc.k23, nk2 = pc.nk2;
    const long long a2x4 = __double_as_longlong(pc.a2x4);   // r2 >= 4a^2 compared on the bit patterns
    const int u0 = uoff[li], u1 = uoff[li + 1];
    const int nt = te - tb;
    const int Rn = nt < int(blockDim.x) ? nt : int(blockDim.x);
    const int G = int(blockDim.x) / Rn;
    const int tl = threadIdx.x % Rn, g = threadIdx.x / Rn;
    for (int i0 = tb; i0 < te; i0 += Rn) {
        const int i = i0 + tl;
        const bool act = i < te && g < G;
        const double xi = act ? pos[i] : 0.0, yi = act ? pos[n + i] : 0.0, zi = act ? pos[2 * n + i] : 0.0;
        double ax = 0, ay = 0, az = 0;   // far pairs, units of s/(8 pi)
        double accd[3] = {0, 0, 0};      // overlapping pairs
        SrcCursor cur{u0, 0};
        while (cur.u < u1) {
            __syncthreads();
            int j = cursor_locate(cur, u1, threadIdx.x, uidx, beg, end);
            sj[threadIdx.x] = j;
            if (j >= 0) {
                sx[threadIdx.x] = pos[j];
                sy[threadIdx.x] = pos[n + j];
                sz[threadIdx.x] = pos[2 * n + j];
                sfx[threadIdx.x] = fs[j];
                sfy[threadIdx.x] = fs[n + j];
                sfz[threadIdx.x] = fs[2 * n + j];
            }
            cur = cursor_advance(cur, u1, int(blockDim.x), uidx, beg, end);
            __syncthreads();
            if (!act) continue;
            for (int jj = g; jj < int(blockDim.x); jj += G) {
                const int jg = sj[jj];
                if (jg < 0) break;
                const double dx = xi - sx[jj], dy = yi - sy[jj], dz = zi - sz[jj];
                const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                const double fx = sfx[jj], fy = sfy[jj], fz = sfz[jj];
                if (__double_as_longlong(r2) >= a2x4) {
                    // [(1 + 2a^2/(3r^2)) F + (1 - 2a^2/r^2)(R.F)/r^2 R] / r = t1 F + t2 R,
                    //   t1 = ri + k23 ri^3,  t2 = ri^3 (1 - 2a^2 ri^2) R.F
                    double ri;
                    if (!rsqrt_seeded(r2, ri)) ri = 1.0 / sqrt(r2);
                    const double ri2 = ri * ri;
                    const double B = ri * ri2;
                    const double t1 = fma(k23, B, ri);
                    const double w = fma(nk2, ri2, 1.0);
                    const double RF = fma(dz, fz, fma(dy, fy, dx * fx));
                    const double t2 = (B * w) * RF;
                    ax = fma(t2, dx, fma(t1, fx, ax));
                    ay = fma(t2, dy, fma(t1, fy, ay));
                    az = fma(t2, dz, fma(t1, fz, az));
                } else if (jg != i) {
                    overlap_pair(dx, dy, dz, r2, fx, fy, fz, a, co, accd);
                }
            }
        }
        __syncthreads();
        red[0][threadIdx.x] = fma(cf, ax, accd[0]);
        red[1][threadIdx.x] = fma(cf, ay, accd[1]);
        red[2][threadIdx.x] = fma(cf, az, accd[2]);
        __syncthreads();
        if (act && g == 0) {
            double v[3];
            for (int c = 0; c < 3; ++c) {
                v[c] = red[c][threadIdx.x];
                for (int gg = 1; gg < G; ++gg) v[c] += red[c][threadIdx.x + gg * Rn];
            }
            const double cs = add_self ? co : 0.0;
            out[3 * size_t(i)] = v[0] + cs * fs[i];
            out[3 * size_t(i) + 1] = v[1] + cs * fs[n + i];
            out[3 * size_t(i) + 2] = v[2] + cs * fs[2 * n + i];
        }
    }
}

// ---------------------------------------------------------------- FP32 form
constexpr int kP32Threads = 256;
constexpr int kP32Chunk = 512;     // sources staged per pass
constexpr int kP32List = 256;      // list boxes per prefix segment
constexpr int kP32Block = 32;      // sources per plain FP32 block between Kahan merges

struct P32Const {
    float a2x4, tiny2, k23, nk2;
    float co_cf, nco_c9, co_c3;   // co_cf = (s/(6 pi a)) / (s/(8 pi)), c9 = 9/(32 a), c3 = 3/(32 a)
};

// Sorted positions as hi + lo floats (x = hi + lo to ~2^-48 relative), so that
// coordinates relative to a leaf centre are formed in FP32 as
// (x_hi - c_hi) + (x_lo - c_lo) with the accuracy of one FP32 rounding of the
// difference; no FP64 work remains in the near-field staging.
__global__ void k_split_f32(const double *pos, int64_t n3, float *p32) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double x = pos[i];
    float hi = float(x);
    p32[i] = hi;
    p32[n3 + i] = float(x - double(hi));
}

int split_positions_f32(Tree &t, cudaStream_t st) {
    int64_t n3 = 3 * t.n;
    k_split_f32<<<unsigned((n3 + 255) / 256), 256, 0, st>>>(t.pos, n3, t.p32);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

// FP64 pair for beads within 1e-3 a of each other (where the FP32 difference of
// coordinates loses the direction), from the FP64 positions.
__device__ __forceinline__ void pair_tiny64(int jg, int i, double a, double co, const double *pos, const double *fs,
                                            int64_t n, double *acc) {
    double ddx = pos[i] - pos[jg], ddy = pos[n + i] - pos[n + jg], ddz = pos[2 * n + i] - pos[2 * n + jg];
    overlap_pair(ddx, ddy, ddz, ddx * ddx + ddy * ddy + ddz * ddz, fs[jg], fs[n + jg], fs[2 * n + jg], a, co, acc);
}

// Hardware reciprocal square root, flushing subnormals (the argument here is at
// least 1e-6 a^2, kept normal by k_pair_const).
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One pair, both branches without divergence, in units of s/(8 pi), with
// ri = 1/max(r, 1e-3 a):
//   r >= 2a          :  t1 = ri + k23 ri^3,      c = ri^3 (1 - 2a^2 ri^2)
//   1e-3 a < r < 2a  :  t1 = co_cf (1 - c9 r),   c = co_cf c3 ri
//   r <= 1e-3 a      :  t1 = c = 0  (the self pair; other such pairs are taken in FP64)
//   u += t1 F + c (R.F) R
__device__ __forceinline__ void pair32(float dx, float dy, float dz, float r2, float fx, float fy, float fz,
                                       const P32Const &k, float &px, float &py, float &pz) {
    const float ri = rsqrt_ftz(fmaxf(r2, k.tiny2));
    const float ri2 = ri * ri;
    const float B = ri * ri2;
    const bool far = r2 >= k.a2x4, on = r2 > k.tiny2;
    float t1 = far ? fmaf(k.k23, B, ri) : fmaf(k.nco_c9, r2 * ri, k.co_cf);
    float c = far ? B * fmaf(k.nk2, ri2, 1.0f) : k.co_c3 * ri;
    t1 = on ? t1 : 0.0f;
    c = on ? c : 0.0f;
    const float t2 = c * fmaf(dz, fz, fmaf(dy, fy, dx * fx));
    px = fmaf(t2, dx, fmaf(t1, fx, px));
    py = fmaf(t2, dy, fmaf(t1, fy, py));
    pz = fmaf(t2, dz, fmaf(t1, fz, pz));
}

// Packed forms over the two targets of a thread (lane .x target a, lane .y
// target b) and one staged source.  x - x_j is formed as x + (-x_j), which
// rounds as the difference does.
__device__ __forceinline__ float2 packed_d(float2 X, float nx0, float nx1) {
    return __fadd2_rn(X, make_float2(nx0, nx1));
}

__device__ __forceinline__ float2 packed_r2(float2 DX, float2 DY, float2 DZ) {
    return __ffma2_rn(DZ, DZ, __ffma2_rn(DY, DY, __fmul2_rn(DX, DX)));
}

// The r >= 2a branch of pair32 on both lanes, for pairs known to be far (the
// clamp and the selects of pair32 are then the identity): the same operations
// in the same order, hence the same rounding lane by lane.
__device__ __forceinline__ void far_packed(float2 DX, float2 DY, float2 DZ, float2 R2, float2 FX, float2 FY,
                                           float2 FZ, float2 K23, float2 NK2, float2 &AX, float2 &AY, float2 &AZ) {
    const float2 RI = make_float2(rsqrt_ftz(R2.x), rsqrt_ftz(R2.y));
    const float2 RI2 = __fmul2_rn(RI, RI);
    const float2 B = __fmul2_rn(RI, RI2);
    const float2 T1 = __ffma2_rn(K23, B, RI);
    const float2 C = __fmul2_rn(B, __ffma2_rn(NK2, RI2, make_float2(1.f, 1.f)));
    const float2 T2 = __fmul2_rn(C, __ffma2_rn(DZ, FZ, __ffma2_rn(DY, FY, __fmul2_rn(DX, FX))));
    AX = __ffma2_rn(T2, DX, __ffma2_rn(T1, FX, AX));
    AY = __ffma2_rn(T2, DY, __ffma2_rn(T1, FY, AY));
    AZ = __ffma2_rn(T2, DZ, __ffma2_rn(T1, FZ, AZ));
}

__device__ __forceinline__ void kahan_merge(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// A leaf of T beads: R = min(ceil(T/2), blockDim) threads per pass carry
// targets i0 + t and i0 + R + t (the two lanes of each packed chain);
// G = blockDim / R groups split every staged chunk.  The U list's boxes are
// prefix-summed in shared memory and each staged bead finds its box by
// binary search.
constexpr int kP32Queue = 256;   // FP64 pairs of one staged chunk handled after its FP32 loop
constexpr size_t kP32Smem = sizeof(float4) * 3 * kP32Chunk + sizeof(int) * kP32Chunk +
                            sizeof(float2) * 6 * kP32Threads + sizeof(double) * 6 * kP32Threads +
                            sizeof(int) * (2 * kP32List + 2) + sizeof(float) * 6 + sizeof(int) * (kP32Queue + 2);

__global__ void __launch_bounds__(kP32Threads, 4) k_p2p32(const int2 *items, const int *leaves, const int *beg,
                                                         const int *end,
                                                         const int *bsys, const double *ctr, const int *uoff,
                                                         const int *uidx, const float *p32, const float *f32,
                                                         const double *pos, const double *fs, int64_t n, SysConst sc,
                                                         int add_self, double *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // staged source e, relative to the target leaf centre, each value twice (both lanes of a
    // packed pair): sS[3e] = (-x, -x, -y, -y), sS[3e+1] = (-z, -z, fx, fx), sS[3e+2] = (fy, fy, fz, fz)
    float4 *sS = reinterpret_cast<float4 *>(smem_raw);
    float2 *sK = reinterpret_cast<float2 *>(sS + 3 * kP32Chunk);   // [6][kP32Threads] Kahan states (S, C)
    double *sD = reinterpret_cast<double *>(sK + 6 * kP32Threads);   // [kP32Threads][6] FP64 pairs
    int *sJ = reinterpret_cast<int *>(sD + 6 * kP32Threads);
    int *lb = sJ + kP32Chunk, *lpre = lb + kP32List;
    float *sCtr = reinterpret_cast<float *>(lpre + kP32List + 2);   // target leaf centre, hi and lo floats
    int *sQn = reinterpret_cast<int *>(sCtr + 6);   // [0] queue length, [1] any FP64 pair in this pass
    int *sQ = sQn + 2;                              // queued pairs: thread << 11 | source slot << 1 | target
    const int2 item = items[blockIdx.x];
    const int li = item.x, b = leaves[li], sys = bsys[b];
    const PairConst &pc = sc.pc[sys];
    const double a = pc.a, cf = pc.cf, co = pc.co;
    P32Const k;
    k.a2x4 = pc.f_a2x4;
    k.tiny2 = pc.f_tiny2;
    k.k23 = pc.f_k23;
    k.nk2 = pc.f_nk2;
    k.co_cf = pc.f_co_cf;
    k.nco_c9 = pc.f_nco_c9;
    k.co_c3 = pc.f_co_c3;
    if (threadIdx.x < 3) {
        const double c = ctr[3 * b + threadIdx.x];
        const float h = float(c);
        sCtr[threadIdx.x] = h;
        sCtr[3 + threadIdx.x] = float(c - double(h));
    }
    if (threadIdx.x == 0) sQn[0] = 0;
    __syncthreads();
    const float chx = sCtr[0], chy = sCtr[1], chz = sCtr[2], clx = sCtr[3], cly = sCtr[4], clz = sCtr[5];
    const float *xh = p32, *yh = p32 + n, *zh = p32 + 2 * n, *xl = p32 + 3 * n, *yl = p32 + 4 * n, *zl = p32 + 5 * n;
    const float2 K23 = make_float2(k.k23, k.k23), NK2 = make_float2(k.nk2, k.nk2);
    const int u0 = uoff[li], u1 = uoff[li + 1];
    const int tb = item.y, te = min(end[b], item.y + kItemTargets), nt = te - tb;
    const int half = (nt + 1) / 2;
    const int Rn = half < kP32Threads ? half : kP32Threads;
    const int G = kP32Threads / Rn;
    const int tl = threadIdx.x % Rn, g = threadIdx.x / Rn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i0 = tb; i0 < te; i0 += 2 * Rn) {
        const int ia = i0 + tl, ib = i0 + Rn + tl;
        const bool act = g < G && ia < te;
        const bool actb = act && ib < te;
        // an absent second target sits far away: its chain stays on the far branch
        const float xa = act ? (xh[ia] - chx) + (xl[ia] - clx) : 0.f;
        const float ya = act ? (yh[ia] - chy) + (yl[ia] - cly) : 0.f;
        const float za = act ? (zh[ia] - chz) + (zl[ia] - clz) : 0.f;
        const float xb = actb ? (xh[ib] - chx) + (xl[ib] - clx) : 1e15f;
        const float yb = actb ? (yh[ib] - chy) + (yl[ib] - cly) : 1e15f;
        const float zb = actb ? (zh[ib] - chz) + (zl[ib] - clz) : 1e15f;
        const float2 X = make_float2(xa, xb), Y = make_float2(ya, yb), Z = make_float2(za, zb);
        for (int c = 0; c < 6; ++c) {
            sK[c * kP32Threads + threadIdx.x] = make_float2(0.f, 0.f);
            sD[6 * threadIdx.x + c] = 0.0;
        }
        if (threadIdx.x == 0) sQn[1] = 0;
        for (int us = u0; us < u1; us += kP32List) {
            const int L = min(kP32List, u1 - us);
            __syncthreads();
            // prefix of the box sizes of this list segment (warp 0)
            if (warp == 0) {
                int carry = 0;
                for (int q0 = 0; q0 < L; q0 += 32) {
                    int q = q0 + lane, cnt = 0;
                    if (q < L) {
                        int C = uidx[us + q];
                        lb[q] = beg[C];
                        cnt = end[C] - beg[C];
                    }
                    int v = cnt;
                    for (int o = 1; o < 32; o <<= 1) {
                        int w = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += w;
                    }
                    if (q < L) lpre[q + 1] = carry + v;
                    carry += __shfl_sync(0xffffffffu, v, 31);
                }
                if (lane == 0) lpre[0] = 0;
            }
            __syncthreads();
            const int Ns = lpre[L];
            for (int c0 = 0; c0 < Ns; c0 += kP32Chunk) {
                const int nS = min(kP32Chunk, Ns - c0);
                // no barrier here: the one after the prefix (first chunk) or after the
                // previous chunk's compute (and its FP64 queue pass) already orders
                // every read of sS and sJ before this chunk's writes
                for (int e = threadIdx.x; e < nS; e += kP32Threads) {
                    int q = c0 + e, lo = 0, hi = L;   // box: lpre[lo] <= q < lpre[lo + 1]
                    while (hi - lo > 1) {
                        int mid = (lo + hi) >> 1;
                        if (lpre[mid] <= q) lo = mid;
                        else hi = mid;
                    }
                    int j = lb[lo] + (q - lpre[lo]);
                    const float px = (xh[j] - chx) + (xl[j] - clx), py = (yh[j] - chy) + (yl[j] - cly),
                                pz = (zh[j] - chz) + (zl[j] - clz);
                    const float fx = f32[j], fy = f32[n + j], fz = f32[2 * n + j];
                    sS[3 * e] = make_float4(-px, -px, -py, -py);
                    sS[3 * e + 1] = make_float4(-pz, -pz, fx, fx);
                    sS[3 * e + 2] = make_float4(fy, fy, fz, fz);
                    sJ[e] = j;
                }
                __syncthreads();
                if (act) {
                    for (int jb = g; jb < nS; jb += kP32Block * G) {
                        const int je = min(nS, jb + kP32Block * G);
                        // accumulators: lane .x for target a, lane .y for target b
                        float2 AX = make_float2(0.f, 0.f), AY = AX, AZ = AX;
                        // both branches with selects per target, and the close-pair queue
                        auto slow = [&](int jj, float2 DX, float2 DY, float2 DZ, float2 R2, float2 FX, float2 FY,
                                        float2 FZ) {
                            pair32(DX.x, DY.x, DZ.x, R2.x, FX.x, FY.x, FZ.x, k, AX.x, AY.x, AZ.x);
                            pair32(DX.y, DY.y, DZ.y, R2.y, FX.x, FY.x, FZ.x, k, AX.y, AY.y, AZ.y);
                            if (!(R2.x > k.tiny2) || !(R2.y > k.tiny2)) {
                                // the self pair, or beads within 1e-3 a: queue all but the self pair
                                const int jg = sJ[jj];
                                if (!(R2.x > k.tiny2) && jg != ia) {
                                    int q = atomicAdd(&sQn[0], 1);
                                    if (q < kP32Queue) sQ[q] = (threadIdx.x << 11) | (jj << 1);
                                }
                                if (actb && !(R2.y > k.tiny2) && jg != ib) {
                                    int q = atomicAdd(&sQn[0], 1);
                                    if (q < kP32Queue) sQ[q] = (threadIdx.x << 11) | (jj << 1) | 1;
                                }
                            }
                        };
                        // Two staged sources per iteration: two independent packed chains.  When
                        // every pair of the lanes running the iteration is far (a warp-uniform
                        // vote), the far branch alone on packed pairs, the same operations as
                        // pair32's far branch lane by lane; otherwise the slow form above.
                        int jj = jb;
                        for (; jj + G < je; jj += 2 * G) {
                            const int j1 = jj + G;
                            const float4 S0 = sS[3 * jj], S1 = sS[3 * jj + 1], S2 = sS[3 * jj + 2];
                            const float4 U0 = sS[3 * j1], U1 = sS[3 * j1 + 1], U2 = sS[3 * j1 + 2];
                            const float2 DX = packed_d(X, S0.x, S0.y), DY = packed_d(Y, S0.z, S0.w),
                                         DZ = packed_d(Z, S1.x, S1.y);
                            const float2 EX = packed_d(X, U0.x, U0.y), EY = packed_d(Y, U0.z, U0.w),
                                         EZ = packed_d(Z, U1.x, U1.y);
                            const float2 R2 = packed_r2(DX, DY, DZ), Q2 = packed_r2(EX, EY, EZ);
                            const float2 FX = make_float2(S1.z, S1.w), FY = make_float2(S2.x, S2.y),
                                         FZ = make_float2(S2.z, S2.w);
                            const float2 GX = make_float2(U1.z, U1.w), GY = make_float2(U2.x, U2.y),
                                         GZ = make_float2(U2.z, U2.w);
                            if (__all_sync(__activemask(), fminf(fminf(R2.x, R2.y), fminf(Q2.x, Q2.y)) >= k.a2x4)) {
                                far_packed(DX, DY, DZ, R2, FX, FY, FZ, K23, NK2, AX, AY, AZ);
                                far_packed(EX, EY, EZ, Q2, GX, GY, GZ, K23, NK2, AX, AY, AZ);
                                continue;
                            }
                            slow(jj, DX, DY, DZ, R2, FX, FY, FZ);
                            slow(j1, EX, EY, EZ, Q2, GX, GY, GZ);
                        }
                        if (jj < je) {
                            const float4 S0 = sS[3 * jj], S1 = sS[3 * jj + 1], S2 = sS[3 * jj + 2];
                            const float2 DX = packed_d(X, S0.x, S0.y), DY = packed_d(Y, S0.z, S0.w),
                                         DZ = packed_d(Z, S1.x, S1.y);
                            const float2 R2 = packed_r2(DX, DY, DZ);
                            const float2 FX = make_float2(S1.z, S1.w), FY = make_float2(S2.x, S2.y),
                                         FZ = make_float2(S2.z, S2.w);
                            if (__all_sync(__activemask(), fminf(R2.x, R2.y) >= k.a2x4))
                                far_packed(DX, DY, DZ, R2, FX, FY, FZ, K23, NK2, AX, AY, AZ);
                            else
                                slow(jj, DX, DY, DZ, R2, FX, FY, FZ);
                        }
                        const float Pv[6] = {AX.x, AY.x, AZ.x, AX.y, AY.y, AZ.y};
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            float2 kc = sK[c * kP32Threads + threadIdx.x];
                            kahan_merge(kc.x, kc.y, Pv[c]);
                            sK[c * kP32Threads + threadIdx.x] = kc;
                        }
                    }
                }
                __syncthreads();
                const int nq = sQn[0];
                if (nq > 0) {
                    // FP64 pairs of this chunk: from the queue, or (queue overflow)
                    // by every thread re-scanning its own sources
                    if (nq <= kP32Queue) {
                        for (int e = threadIdx.x; e < nq; e += kP32Threads) {
                            const int v = sQ[e], t = v >> 11, jj = (v >> 1) & 1023, h = v & 1;
                            const int i = i0 + (t % Rn) + h * Rn;
                            double acc[3] = {0, 0, 0};
                            pair_tiny64(sJ[jj], i, a, co, pos, fs, n, acc);
                            for (int c = 0; c < 3; ++c) atomicAdd(&sD[6 * t + 3 * h + c], acc[c]);
                        }
                    } else if (act) {
                        for (int jj = g; jj < nS; jj += G) {
                            const float4 S0 = sS[3 * jj], S1 = sS[3 * jj + 1];
                            const int jg = sJ[jj];
                            for (int h = 0; h < 2; ++h) {
                                const float dx = (h ? xb : xa) + S0.x, dy = (h ? yb : ya) + S0.z, dz = (h ? zb : za) + S1.x;
                                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                const int i = h ? ib : ia;
                                if (!(r2 > k.tiny2) && jg != i && (h == 0 || actb))
                                    pair_tiny64(jg, i, a, co, pos, fs, n, &sD[6 * threadIdx.x + 3 * h]);
                            }
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        sQn[0] = 0;
                        sQn[1] = 1;
                    }
                }
            }
        }
        // group reduction: one thread per (target, component) merges the Kahan
        // states (S, C) of the G groups in FP32 (Kahan over the S, plain sum of
        // the small C) and forms the FP64 result once
        __syncthreads();
        const bool tiny = sQn[1] != 0;   // read before the barrier: the next pass resets it after
        __syncthreads();
        for (int q = threadIdx.x; q < 6 * Rn; q += kP32Threads) {
            const int hc = q / Rn, tt = q - hc * Rn, h = hc / 3, c = hc - 3 * h;
            const int i = i0 + h * Rn + tt;
            if (i < te) {
                float S = 0.f, C = 0.f, Cs = 0.f;
                for (int gg = 0; gg < G; ++gg) {
                    const float2 v = sK[hc * kP32Threads + tt + gg * Rn];
                    kahan_merge(S, C, v.x);
                    Cs += v.y;
                }
                double u = cf * (double(S) - (double(C) + double(Cs)));
                if (tiny)
                    for (int gg = 0; gg < G; ++gg) u += sD[6 * (tt + gg * Rn) + 3 * h + c];
                out[3 * size_t(i) + c] = u + (add_self ? co * fs[c * n + i] : 0.0);
            }
        }
        __syncthreads();   // the next pass clears sK and sD
    }
}

// The dynamic shared memory of k_p2p32 exceeds the default 48 KB: raise the
// limit once per device.
static cudaError_t set_p2p32_smem() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(dev)) return cudaSuccess;
    e = cudaFuncSetAttribute(k_p2p32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kP32Smem));
    if (e == cudaSuccess) done.insert(dev);
    return e;
}

// U lists (near field, self term added), the direct substitutes of small
// W / X interactions (no self term), or both in one pass (the full matvec).
int run_p2p(Tree &t, const double *fs, double *out, const SysConst &sc, cudaStream_t st, int list) {
    const bool direct_list = list == kListD, merged = list == kListM;
    const int *off = merged ? t.m_off : (direct_list ? t.d_off : t.u_off);
    const int *idx = merged ? t.m_idx : (direct_list ? t.d_idx : t.u_idx);
    int add_self = direct_list ? 0 : 1;
    const int2 *items = merged ? t.m_items : (direct_list ? t.d_items : t.u_items);
    if (t.n_items == 0) return RPY_OK;
    if (t.params.precision == RPY_FP32) {
        RPY_CHECK(set_p2p32_smem());
        k_p2p32<<<t.n_items, kP32Threads, kP32Smem, st>>>(items, t.leaves, t.b_begin, t.b_end, t.b_sys, t.b_center,
                                                          off, idx, t.p32, t.f32, t.pos, fs, t.n, sc, add_self, out);
        RPY_LAUNCHED(1);
    } else {
        k_p2p<<<t.n_items, kP2PThreads, 0, st>>>(items, t.leaves, t.b_begin, t.b_end, t.b_sys, off, idx, t.pos, fs,
                                                 t.n, sc, add_self, out);
        RPY_LAUNCHED(1);
    }
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

}  // namespace rpy
