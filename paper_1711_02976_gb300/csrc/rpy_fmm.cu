// Far field of the RPY matvec: the four Laplace potentials of Sec. 2 through
// an adaptive FMM whose multipole-to-local step runs on plane-wave
// (exponential) expansions (M-to-I, I-to-I, I-to-L of Fig. "op").
//
// Charge sets (Sec. 2): q_1..q_3 = F^1..F^3, q_4 = F . (r - c0) with c0 the
// centre of the system's bounding cube (Eq. 2.8 holds for any common origin).
//
// Kernels, in launch order:
//   k_p2m      S->M   leaves: M_n^m = sum_j q_j conj(y_n^m(eta_j))
//   k_m2m_child, k_m2m_sum  M->M   per child: rotate to the shift axis, z-shift, rotate back;
//                      per parent: add the children's shares in octant order
//   k_m2x      M->I   rotate into the frame of each axis, outgoing plane waves
//                     W_kj = (w_k/M_k) sum_{n,m} M_n^m i^|m| lambda_k^n e^{i m a_kj} / sqrt((n-|m|)!(n+|m|)!)
//   k_x2x      I->I   merge-and-shift: per parent and direction, sources are
//                     shifted to the parent centre and summed per group of
//                     targets they serve, then shifted once to each child
//   k_x2l      I->L   L_n^m = i^|m| sum_k (-lambda_k)^n / sqrt(...) sum_j I_kj e^{-i m a_kj},
//                     rotated back to the world frame
//   k_p2l      S->L   X list
//   k_l2l_rot  L->L   the same for locals, level by level downward
//   k_far_eval L->T, M->T   L2P for the leaf and M2P for its W list, with the
//                     gradients and Hessians of Theorems 1-2 formed as
//                     derivative expansions per box, combined by Eq. (2.8):
//                     u = C1 [L1 L2 L3] - C1 sum_k x_k grad L_k + C1 grad L4 - C2 grad L_C.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>

#include "rpy_harmonics.h"

namespace rpy {

__device__ __forceinline__ int deg_of(int idx) {
    int n = int((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
    while (tri(n + 1, 0) <= idx) ++n;
    while (tri(n, 0) > idx) --n;
    return n;
}

// ---------------------------------------------------------------- harmonics, several points per warp
// Lanes per point: columns m and P - m share a lane, so every lane runs P + 2
// recurrence steps (a column per lane would leave the lanes of high m idle
// while column 0 runs P + 1 steps, and lanes above P idle altogether; the
// FP64 pipe is charged per warp instruction).
__host__ __device__ constexpr int harm_lanes(int P) { return P / 2 + 1; }

// Solid harmonics (regular, or irregular when IRREG) of one point into out[],
// columns c and P - c of it.
template <typename T, bool IRREG>
__device__ void lane_harmonics(T x, T y, T z, int P, const T *ra, const T *rb, const T *cm, cpx<T> *out, int c) {
    const T r2 = fma(z, z, fma(y, y, x * x));
    const T ir2 = IRREG ? T(1) / r2 : T(0);
    const cpx<T> w = IRREG ? mk(x * ir2, y * ir2) : mk(x, y);
    const T d0 = IRREG ? sqrt(ir2) : T(1);
    const T zz = IRREG ? z * ir2 : z;   // factor of the a-coefficients
    const T rr = IRREG ? ir2 : r2;      // factor of the b-coefficients
    for (int h = 0; h < 2; ++h) {
        const int m = h ? P - c : c;
        if (h && m == c) break;
        cpx<T> pw = mk<T>(1, 0), base = w;   // w^m by binary powering
        for (int e = m; e; e >>= 1) {
            if (e & 1) pw = pw * base;
            base = base * base;
        }
        const T s0 = cm[m] * d0;
        cpx<T> p1 = mk(s0 * pw.x, s0 * pw.y), p2 = mk<T>(0, 0);
        out[tri(m, m)] = p1;
        for (int n = m + 1; n <= P; ++n) {
            const int i = tri(n, m);
            const T A = ra[i] * zz, B = rb[i] * rr;
            const cpx<T> cn = mk(fma(A, p1.x, -B * p2.x), fma(A, p1.y, -B * p2.y));
            out[i] = cn;
            p2 = p1;
            p1 = cn;
        }
    }
}

// Streaming per-thread evaluation of NE real fields f_q = sum_{n<=P,m} w_m Re(E_q[n,m] h_n^m(v)),
// w_0 = 1, w_m = 2 (m > 0); W2: the coefficients already carry w_m.
template <typename T, int NE, bool IRREG, bool W2 = false>
__device__ void eval_fields(T x, T y, T z, int P, const cpx<T> *E, int stride, const T *ra, const T *rb,
                            const T *rc, T *acc) {
    const T r2 = fma(z, z, fma(y, y, x * x));
    const T ir2 = IRREG ? T(1) / r2 : T(0);
    const cpx<T> w = IRREG ? mk(x * ir2, y * ir2) : mk(x, y);
    const T zz = IRREG ? z * ir2 : z;
    const T rr = IRREG ? ir2 : r2;
    cpx<T> diag = IRREG ? mk<T>(sqrt(ir2), 0) : mk<T>(1, 0);
    for (int m = 0; m <= P; ++m) {
        if (m > 0) diag = rc[m] * (w * diag);
        const T wm = (W2 || m == 0) ? T(1) : T(2);
        cpx<T> p2 = mk<T>(0, 0), p1 = diag;
        {
            const int i = tri(m, m);
            const cpx<T> hw = W2 ? diag : mk(wm * diag.x, wm * diag.y);
#pragma unroll
            for (int q = 0; q < NE; ++q) {
                const cpx<T> e = E[q * stride + i];
                acc[q] = fma(-e.y, hw.y, fma(e.x, hw.x, acc[q]));
            }
        }
        for (int n = m + 1; n <= P; ++n) {
            const int i = tri(n, m);
            const T A = ra[i] * zz, B = rb[i] * rr;
            const cpx<T> c = mk(fma(A, p1.x, -B * p2.x), fma(A, p1.y, -B * p2.y));
            const cpx<T> hw = W2 ? c : mk(wm * c.x, wm * c.y);
#pragma unroll
            for (int q = 0; q < NE; ++q) {
                const cpx<T> e = E[q * stride + i];
                acc[q] = fma(-e.y, hw.y, fma(e.x, hw.x, acc[q]));
            }
            p2 = p1;
            p1 = c;
        }
    }
}

// ---------------------------------------------------------------- derivative expansions
// Real-field derivative expansions (ladder relations of Sec. 2, Theorems 1-2),
// computed by the whole CTA.  src: degree ps coefficients.  dst: x, y, z
// derivatives, each zero-padded to stride.
template <typename T>
struct Lad {
    const T *lz, *lp, *lq, *mz, *mp, *mq;
};

template <typename T>
__device__ void d_local(const cpx<T> *src, int ps, cpx<T> *dx, cpx<T> *dy, cpx<T> *dz, int P, const Lad<T> &G) {
    // degree k <= ps-1 from L_{k+1}
    for (int i = threadIdx.x; i < ncoef(P); i += blockDim.x) {
        int k = deg_of(i), m = i - tri(k, 0);
        cpx<T> X = mk<T>(0, 0), Y = X, Z = X;
        if (k <= ps - 1) {
            Z = G.lz[i] * src[tri(k + 1, m)];
            cpx<T> Pv = m >= 1 ? G.lp[i] * src[tri(k + 1, m - 1)] : (-G.lq[i]) * conj(src[tri(k + 1, 1)]);
            cpx<T> Qv = (-G.lq[i]) * src[tri(k + 1, m + 1)];
            X = mk(T(0.5) * (Pv.x + Qv.x), T(0.5) * (Pv.y + Qv.y));
            Y = mk(T(0.5) * (Pv.y - Qv.y), T(-0.5) * (Pv.x - Qv.x));
        }
        dx[i] = X;
        dy[i] = Y;
        dz[i] = Z;
    }
}

template <typename T>
__device__ void d_multipole(const cpx<T> *src, int ps, cpx<T> *dx, cpx<T> *dy, cpx<T> *dz, int P, const Lad<T> &G) {
    // degree k <= ps+1 from M_{k-1}
    for (int i = threadIdx.x; i < ncoef(P); i += blockDim.x) {
        int k = deg_of(i), m = i - tri(k, 0);
        cpx<T> X = mk<T>(0, 0), Y = X, Z = X;
        if (k >= 1 && k <= ps + 1) {
            if (m <= k - 1) Z = (-G.mz[i]) * src[tri(k - 1, m)];
            cpx<T> Pv = mk<T>(0, 0), Qv = mk<T>(0, 0);
            if (m >= 1) Pv = G.mp[i] * src[tri(k - 1, m - 1)];
            else if (k >= 2) Pv = (-G.mp[i]) * conj(src[tri(k - 1, 1)]);
            if (m + 1 <= k - 1) Qv = (-G.mq[i]) * src[tri(k - 1, m + 1)];
            X = mk(T(0.5) * (Pv.x + Qv.x), T(0.5) * (Pv.y + Qv.y));
            Y = mk(T(0.5) * (Pv.y - Qv.y), T(-0.5) * (Pv.x - Qv.x));
        }
        dx[i] = X;
        dy[i] = Y;
        dz[i] = Z;
    }
}

// Coefficient i of one component c (0 = x, 1 = y, 2 = z) of the gradient of a
// local (d_loc_one) or multipole (d_mul_one) expansion of degree ps: the
// single-output forms of d_local and d_multipole.
template <typename T>
__device__ __forceinline__ cpx<T> d_loc_one(const cpx<T> *src, int ps, int c, int i, const Lad<T> &G) {
    const int k = deg_of(i), m = i - tri(k, 0);
    if (k > ps - 1) return mk<T>(0, 0);
    if (c == 2) return G.lz[i] * src[tri(k + 1, m)];
    const cpx<T> Pv = m >= 1 ? G.lp[i] * src[tri(k + 1, m - 1)] : (-G.lq[i]) * conj(src[tri(k + 1, 1)]);
    const cpx<T> Qv = (-G.lq[i]) * src[tri(k + 1, m + 1)];
    return c == 0 ? mk(T(0.5) * (Pv.x + Qv.x), T(0.5) * (Pv.y + Qv.y))
                  : mk(T(0.5) * (Pv.y - Qv.y), T(-0.5) * (Pv.x - Qv.x));
}

template <typename T>
__device__ __forceinline__ cpx<T> d_mul_one(const cpx<T> *src, int ps, int c, int i, const Lad<T> &G) {
    const int k = deg_of(i), m = i - tri(k, 0);
    if (k < 1 || k > ps + 1) return mk<T>(0, 0);
    if (c == 2) return m <= k - 1 ? (-G.mz[i]) * src[tri(k - 1, m)] : mk<T>(0, 0);
    cpx<T> Pv = mk<T>(0, 0), Qv = mk<T>(0, 0);
    if (m >= 1) Pv = G.mp[i] * src[tri(k - 1, m - 1)];
    else if (k >= 2) Pv = (-G.mp[i]) * conj(src[tri(k - 1, 1)]);
    if (m + 1 <= k - 1) Qv = (-G.mq[i]) * src[tri(k - 1, m + 1)];
    return c == 0 ? mk(T(0.5) * (Pv.x + Qv.x), T(0.5) * (Pv.y + Qv.y))
                  : mk(T(0.5) * (Pv.y - Qv.y), T(-0.5) * (Pv.x - Qv.x));
}

// ---------------------------------------------------------------- table access
template <typename T>
struct Rec {
    const T *a, *b, *c, *cm;
};

template <typename T>
__device__ Rec<T> load_rec(const DevTables<T> &D, T *sm) {
    int P = D.p + 2;
    int nc = ncoef(P);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        sm[i] = D.rec_a[i];
        sm[nc + i] = D.rec_b[i];
    }
    for (int i = threadIdx.x; i <= P; i += blockDim.x) {
        sm[2 * nc + i] = D.rec_c[i];
        sm[2 * nc + P + 1 + i] = D.rec_cm[i];
    }
    Rec<T> r{sm, sm + nc, sm + 2 * nc, sm + 2 * nc + P + 1};
    return r;
}

// ladder tables follow the recurrence tables in shared memory
template <typename T>
__device__ Lad<T> load_lad(const DevTables<T> &D, T *sm) {
    int nl = ncoef(D.p + 2);
    for (int i = threadIdx.x; i < 6 * nl; i += blockDim.x) sm[i] = D.lad[i];
    Lad<T> g{sm, sm + nl, sm + 2 * nl, sm + 3 * nl, sm + 4 * nl, sm + 5 * nl};
    return g;
}

template <typename T>
__host__ __device__ inline int rec_floats(int p) {
    return 2 * ncoef(p + 2) + 2 * (p + 3);
}

template <typename T>
__host__ __device__ inline int tab_floats(int p) {   // recurrences + ladders, rounded to an even count
    return ((rec_floats<T>(p) + 6 * ncoef(p + 2)) + 1) & ~1;
}


// ---------------------------------------------------------------- P2M / P2L

// Beads per chunk of P2M / P2L: one round of harmonics, (warps x points per warp).
__host__ __device__ inline int p2x_chunk(int p, int threads) { return (threads / 32) * (32 / harm_lanes(p)); }

// MODE 0: P2M over the leaf's own beads (multipole about its centre)
// MODE 1: P2L over the beads of every box in X(b) (local about b's centre)
// The fourth charge q4 = F . (r - o) takes its origin o at the expansion's own
// centre when rb is set (box origin), else at the system's cube centre.
template <typename T, int MODE>
__global__ void k_p2x(int b0, int nb, DevTables<T> D, const int *beg, const int *end, const double *ctr,
                      const double *side, const int *lvl, const int *leaf, const int *bsys, const int *xoff,
                      const int *xidx, const double *pos, const double *fs, const double *lapq, int64_t n,
                      SysConst sc, cpx<T> *out, int rb) {
    const int kChunkB = p2x_chunk(D.p, blockDim.x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    if (b >= b0 + nb) return;
    if (lvl[b] < 2) return;
    if (MODE == 0 && !leaf[b]) return;
    int nsrc = MODE == 0 ? 1 : xoff[b + 1] - xoff[b];
    if (nsrc == 0) return;
    const int p = D.p, nc = ncoef(p);
    T *smr = reinterpret_cast<T *>(smem_raw);
    Rec<T> R = load_rec(D, smr);
    cpx<T> *ybuf = reinterpret_cast<cpx<T> *>(smr + ((rec_floats<T>(p) + 1) & ~1));
    cpx<T> *acc = ybuf + kChunkB * nc;
    cpx<T> *cmp = acc + kSets * nc;   // FP32: compensation of the running sums
    T *q = reinterpret_cast<T *>(cmp + kSets * nc);
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) acc[i] = cmp[i] = mk<T>(0, 0);
    int sy = bsys[b];
    double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2];
    const double c0x = rb ? cx : sc.cube[4 * sy], c0y = rb ? cy : sc.cube[4 * sy + 1],
                 c0z = rb ? cz : sc.cube[4 * sy + 2];   // origin of q4
    const double ih = sc.pc[sy].icube * pow2i(lvl[b]);   // 1 / side[b], exactly
    int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // harmonics: hG points per warp, lane -> (point hg, column pair hc)
    const int hL = harm_lanes(p), hG = 32 / hL, hg = (threadIdx.x & 31) / hL, hc = (threadIdx.x & 31) - hg * hL;
    __syncthreads();
    for (int si = 0; si < nsrc; ++si) {
        int src = MODE == 0 ? b : xidx[xoff[b] + si];
        int j0 = beg[src], j1 = end[src];
        for (int jc = j0; jc < j1; jc += kChunkB) {
            int cnt = min(kChunkB, j1 - jc);
            for (int t0 = warp * hG; t0 < cnt; t0 += nwarp * hG) {
                const int t = t0 + hg;
                if (hg < hG && t < cnt) {
                    int j = jc + t;
                    T ex = T((pos[j] - cx) * ih), ey = T((pos[n + j] - cy) * ih), ez = T((pos[2 * n + j] - cz) * ih);
                    lane_harmonics<T, MODE == 1>(ex, ey, ez, p, R.a, R.b, R.cm, ybuf + t * nc, hc);
                }
            }
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                int j = jc + t;
                if (lapq) {
                    for (int k = 0; k < kSets; ++k) q[4 * t + k] = T(lapq[4 * j + k]);
                } else {
                    double fx = fs[j], fy = fs[n + j], fz = fs[2 * n + j];
                    q[4 * t] = T(fx);
                    q[4 * t + 1] = T(fy);
                    q[4 * t + 2] = T(fz);
                    q[4 * t + 3] = T(fx * (pos[j] - c0x) + fy * (pos[n + j] - c0y) + fz * (pos[2 * n + j] - c0z));
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
                int k = e / nc, i = e - k * nc;
                cpx<T> a = sizeof(T) == 4 ? mk<T>(0, 0) : acc[e];
                for (int t = 0; t < cnt; ++t) {
                    cpx<T> yv = ybuf[t * nc + i];
                    T qq = q[4 * t + k];
                    a.x += qq * yv.x;
                    a.y -= qq * yv.y;   // conj
                }
                if constexpr (sizeof(T) == 4) {
                    // a leaf (or an X-list source) may hold hundreds to thousands of beads: the
                    // chunk's plain sum enters the running sum by compensated (Kahan) addition
                    cpx<T> sum = acc[e], c = cmp[e];
                    const T yx = a.x - c.x, tx = sum.x + yx;
                    c.x = (tx - sum.x) - yx;
                    sum.x = tx;
                    const T yy = a.y - c.y, ty = sum.y + yy;
                    c.y = (ty - sum.y) - yy;
                    sum.y = ty;
                    acc[e] = sum;
                    cmp[e] = c;
                } else {
                    acc[e] = a;
                }
            }
            __syncthreads();
        }
    }
    cpx<T> *o = out + size_t(b) * kSets * nc;
    for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
        if (MODE == 0) o[e] = acc[e];
        else o[e] += acc[e];
    }
}

// ---------------------------------------------------------------- M2M / L2L

// Dense per-octant operators (used by the FP32 form, where one streaming pass
// over the operator beats the rotation's extra synchronisation).
// M2M: parent M = sum over children of T_o [child M]; output degree n uses inputs of degree <= n.
// rb (box origin of q4): the child's set 4 moves its origin from the child's
// centre to the parent's first, M4 += (c_child - c_parent) . M_F (sets 1..3).
template <typename T>
__global__ void k_m2m(int b0, int nb, DevTables<T> D, const int *leaf, const int *child, const double *side,
                      int rb, cpx<T> *M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    if (leaf[b]) return;
    const int nc = ncoef(D.p), Dd = 2 * nc;
    T *X = reinterpret_cast<T *>(smem_raw);
    int r = threadIdx.x;
    int kmax = r < Dd ? 2 * ncoef(deg_of(r >> 1)) : 0;
    T acc[kSets] = {0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
        int c = child[8 * b + o];
        if (c < 0) continue;
        const T *src = reinterpret_cast<const T *>(M + size_t(c) * kSets * nc);
        __syncthreads();
        for (int i = threadIdx.x; i < kSets * Dd; i += blockDim.x) X[i] = src[i];
        __syncthreads();
        if (rb) {
            const double h = 0.5 * side[c];   // child centre - parent centre = h (2 bit - 1) per axis
            const T dx = T((o & 1) ? h : -h), dy = T((o & 2) ? h : -h), dz = T((o & 4) ? h : -h);
            for (int i = threadIdx.x; i < Dd; i += blockDim.x)
                X[3 * Dd + i] = fma(dz, X[2 * Dd + i], fma(dy, X[Dd + i], fma(dx, X[i], X[3 * Dd + i])));
            __syncthreads();
        }
        if (r < Dd) {
            const T *Tt = D.m2m_t + size_t(o) * Dd * Dd;
            for (int k = 0; k < kmax; ++k) {
                T t = Tt[size_t(k) * Dd + r];
#pragma unroll
                for (int s = 0; s < kSets; ++s) acc[s] += t * X[s * Dd + k];
            }
        }
    }
    if (r < Dd) {
        T *dst = reinterpret_cast<T *>(M + size_t(b) * kSets * nc);
        for (int s = 0; s < kSets; ++s) dst[s * Dd + r] = acc[s];
    }
}

// L2L: child L += S_o [parent L]; output degree k uses inputs of degree >= k.
// rb (box origin of q4): the shifted set 4 moves its origin from the parent's
// centre to the child's, L4 += (c_parent - c_child) . L_F.
template <typename T>
__global__ void k_l2l(int b0, int nb, DevTables<T> D, const int *par, const int *cell, const double *side, int rb,
                      cpx<T> *L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    int P = par[b];
    const int nc = ncoef(D.p), Dd = 2 * nc;
    T *X = reinterpret_cast<T *>(smem_raw);
    const T *src = reinterpret_cast<const T *>(L + size_t(P) * kSets * nc);
    for (int i = threadIdx.x; i < kSets * Dd; i += blockDim.x) X[i] = src[i];
    __syncthreads();
    int r = threadIdx.x;
    if (r >= Dd) return;
    int o = (cell[3 * b] & 1) | ((cell[3 * b + 1] & 1) << 1) | ((cell[3 * b + 2] & 1) << 2);
    int kdeg = deg_of(r >> 1);
    int k0 = 2 * tri(kdeg, 0);
    const T *St = D.l2l_t + size_t(o) * Dd * Dd;
    T acc[kSets] = {0, 0, 0, 0};
    for (int k = k0; k < Dd; ++k) {
        T t = St[size_t(k) * Dd + r];
#pragma unroll
        for (int s = 0; s < kSets; ++s) acc[s] += t * X[s * Dd + k];
    }
    if (rb) {
        const double h = 0.5 * side[b];   // parent centre - child centre = -h (2 bit - 1) per axis
        const T dx = T((o & 1) ? -h : h), dy = T((o & 2) ? -h : h), dz = T((o & 4) ? -h : h);
        acc[3] = fma(dz, acc[2], fma(dy, acc[1], fma(dx, acc[0], acc[3])));
    }
    T *dst = reinterpret_cast<T *>(L + size_t(b) * kSets * nc);
    for (int s = 0; s < kSets; ++s) dst[s * Dd + r] += acc[s];
}

// ---------------------------------------------------------------- rotations
// dst[s] = R src[s] per degree block (real 2-layout, block size 2(n+1)).
// The factorized rotation of the four sets: tmp <- za (src) (one 2x2 rotation per
// coefficient), then dst <- zc (Y tmp), Y acting on real and imaginary parts
// separately.  src and dst may not alias tmp; the caller synchronises after.
template <typename T, bool QUARTER = false>
__device__ void rotate_sets_f(const T *rf, const int *foff, int p, const cpx<T> *src, cpx<T> *tmp, cpx<T> *dst) {
    const int nc = ncoef(p);
    for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
        const int st = e / nc, i = e - st * nc, n = deg_of(i), m = i - tri(n, 0);
        const T *za = rf + foff[n];
        const T c = za[2 * m], sn = za[2 * m + 1];
        const cpx<T> v = src[st * nc + i];
        tmp[e] = mk(fma(c, v.x, -sn * v.y), fma(sn, v.x, c * v.y));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
        const int st = e / nc, i = e - st * nc, n = deg_of(i), m = i - tri(n, 0), q = n + 1;
        const T *o = rf + foff[n];
        const T *yre = o + 4 * q + m * q, *yim = o + 4 * q + q * q + m * q;
        const cpx<T> *in = tmp + st * nc + tri(n, 0);
        T re = 0, im = 0;
        if (QUARTER) {
            // middle angle pi/2 (the frame rotations): the y blocks are checkerboards
            // (checked when the tables are built); Im of m = 0 is zero for real fields
            for (int k = (m + n) & 1; k < q; k += 2) re = fma(yre[k], in[k].x, re);
            if (m > 0)
                for (int k = 1 + ((m + n) & 1); k < q; k += 2) im = fma(yim[k], in[k].y, im);
        } else {
            for (int k = 0; k < q; ++k) {
                re = fma(yre[k], in[k].x, re);
                im = fma(yim[k], in[k].y, im);
            }
        }
        const T c = o[2 * q + 2 * m], sn = o[2 * q + 2 * m + 1];
        dst[st * nc + i] = mk(fma(c, re, -sn * im), fma(sn, re, c * im));
    }
}

// ---------------------------------------------------------------- rotation-based M2M / L2L
// Child octant o: rotate into the frame whose z axis is the shift direction,
// apply the m-diagonal z-shift, rotate back (O(p^3) per child instead of the
// O(p^4) dense operator).
// One child per block (the children of one level): rotate into the frame
// whose z axis is the shift direction, apply the m-diagonal z-shift, rotate back
// (O(p^3) per child instead of the O(p^4) dense operator), and write the
// child's share to its slot Sc[parent][octant]; k_m2m_sum adds the slots of each
// parent in octant order (a fixed order: the result does not depend on timing).
// rb (box origin of q4): the share's set 4 moves its origin from the child's
// centre to the parent's, M4 += (c_child - c_parent) . M_F.
template <typename T>
__global__ void k_m2m_child(int c0, int pb0, DevTables<T> D, const int *par, const int *cell, const double *side,
                            int rb, const cpx<T> *M, cpx<T> *Sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = c0 + blockIdx.x;
    const int p = D.p, nc = ncoef(p), P1 = p + 1;
    cpx<T> *X = reinterpret_cast<cpx<T> *>(smem_raw);
    cpx<T> *Y = X + kSets * nc;
    cpx<T> *Tm = Y + kSets * nc;   // rotation scratch
    const int o = (cell[3 * c] & 1) | ((cell[3 * c + 1] & 1) << 1) | ((cell[3 * c + 2] & 1) << 2);
    const cpx<T> *src = M + size_t(c) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) X[i] = src[i];
    __syncthreads();
    rotate_sets_f(D.forot_fwd + size_t(o) * D.frot_len, D.frot_off, p, X, Tm, Y);
    __syncthreads();
    for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
        int st = e / nc, i = e - st * nc;
        int n = deg_of(i), m = i - tri(n, 0);
        const T *z = D.zm2m + size_t(i) * P1;
        cpx<T> a = mk<T>(0, 0);
        for (int k = m; k <= n; ++k) a += z[k] * Y[st * nc + tri(k, m)];
        X[e] = a;
    }
    __syncthreads();
    rotate_sets_f(D.forot_bwd + size_t(o) * D.frot_len, D.frot_off, p, X, Tm, Y);
    __syncthreads();
    cpx<T> *dst = Sc + (size_t(par[c] - pb0) * 8 + o) * kSets * nc;
    const double h = 0.5 * side[c];
    const T dx = T((o & 1) ? h : -h), dy = T((o & 2) ? h : -h), dz = T((o & 4) ? h : -h);
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) {
        cpx<T> v = Y[i];
        if (rb && i >= 3 * nc) {
            const int k = i - 3 * nc;
            const cpx<T> fx = Y[k], fy = Y[nc + k], fz = Y[2 * nc + k];
            v = mk(fma(dz, fz.x, fma(dy, fy.x, fma(dx, fx.x, v.x))), fma(dz, fz.y, fma(dy, fy.y, fma(dx, fx.y, v.y))));
        }
        dst[i] = v;
    }
}

template <typename T>
__global__ void k_m2m_sum(int b0, int nc4, const int *leaf, const int *child, const cpx<T> *Sc, cpx<T> *M) {
    const int b = b0 + blockIdx.x;
    if (leaf[b]) return;
    int ch[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) ch[o] = child[8 * b + o];
    const cpx<T> *src = Sc + size_t(blockIdx.x) * 8 * nc4;
    for (int i = threadIdx.x; i < nc4; i += blockDim.x) {
        cpx<T> acc = mk<T>(0, 0);
#pragma unroll
        for (int o = 0; o < 8; ++o)
            if (ch[o] >= 0) acc += src[size_t(o) * nc4 + i];
        M[size_t(b) * nc4 + i] = acc;
    }
}

// rb (box origin of q4): the shifted set 4 moves its origin from the parent's
// centre to the child's, L4 += (c_parent - c_child) . L_F.
template <typename T>
__global__ void k_l2l_rot(int b0, int nb, DevTables<T> D, const int *par, const int *cell, const double *side,
                          int rb, cpx<T> *L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    int P = par[b];
    const int p = D.p, nc = ncoef(p), P1 = p + 1;
    cpx<T> *X = reinterpret_cast<cpx<T> *>(smem_raw);
    cpx<T> *Y = X + kSets * nc;
    cpx<T> *Tm = Y + kSets * nc;   // rotation scratch
    int o = (cell[3 * b] & 1) | ((cell[3 * b + 1] & 1) << 1) | ((cell[3 * b + 2] & 1) << 2);
    const cpx<T> *src = L + size_t(P) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) X[i] = src[i];
    __syncthreads();
    rotate_sets_f(D.forot_fwd + size_t(o) * D.frot_len, D.frot_off, p, X, Tm, Y);
    __syncthreads();
    for (int e = threadIdx.x; e < kSets * nc; e += blockDim.x) {
        int st = e / nc, i = e - st * nc;
        int n = deg_of(i), m = i - tri(n, 0);
        const T *z = D.zl2l + size_t(i) * P1;
        cpx<T> a = mk<T>(0, 0);
        for (int k = n; k <= p; ++k) a += z[k] * Y[st * nc + tri(k, m)];
        X[e] = a;
    }
    __syncthreads();
    rotate_sets_f(D.forot_bwd + size_t(o) * D.frot_len, D.frot_off, p, X, Tm, Y);
    __syncthreads();
    cpx<T> *dst = L + size_t(b) * kSets * nc;
    const double h = 0.5 * side[b];
    const T dx = T((o & 1) ? -h : h), dy = T((o & 2) ? -h : h), dz = T((o & 4) ? -h : h);
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) {
        cpx<T> v = Y[i];
        if (rb && i >= 3 * nc) {
            const int k = i - 3 * nc;
            const cpx<T> fx = Y[k], fy = Y[nc + k], fz = Y[2 * nc + k];
            v = mk(fma(dz, fz.x, fma(dy, fy.x, fma(dx, fx.x, v.x))), fma(dz, fz.y, fma(dy, fy.y, fma(dx, fx.y, v.y))));
        }
        dst[i] += v;
    }
}

// ---------------------------------------------------------------- M2X
template <typename T>
__global__ void k_m2x(int b0, int nb, DevTables<T> D, const cpx<T> *M, cpx<T> *Xo, int f0, int nf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    const int p = D.p, nc = ncoef(p), s = D.s, S = D.S, P1 = p + 1;
    // A per node k: [P1][4 sets] at stride NS = 4 P1 + 1, so that the units of
    // neighbouring nodes in one warp read different shared-memory banks
    const int NS = kSets * P1 + 1;
    cpx<T> *Mw = reinterpret_cast<cpx<T> *>(smem_raw);
    cpx<T> *Mf = Mw + kSets * nc;
    cpx<T> *AE = Mf + kSets * nc;       // [s][NS]
    cpx<T> *AO = AE + s * NS;
    cpx<T> *Tm = AO + s * NS;           // rotation scratch
    const cpx<T> *src = M + size_t(b) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Mw[i] = src[i];
    __syncthreads();
    size_t base = size_t(b) * (2 * nf) * kSets * S;   // frames f0 .. f0 + nf - 1 of this pass
    const int hP = harm_lanes(p);
    for (int f = f0; f < f0 + nf; ++f) {
        const cpx<T> *Mu = Mw;
        if (f > 0) {
            rotate_sets_f<T, true>(D.frot_fwd + size_t(f - 1) * D.frot_len, D.frot_off, p, Mw, Tm, Mf);
            __syncthreads();
            Mu = Mf;
        }
        // A_k^m split by parity of n + m (the - direction is the reflection (-1)^{n+m}),
        // stored as 2 i^m A_k^m so that the wave sum below needs no sign logic:
        // even m feed the real part, odd m the imaginary part.  One thread per
        // (set, node k, column pair (m, p - m)): p + 2 terms each.
        for (int e = threadIdx.x; e < kSets * s * hP; e += blockDim.x) {
            const int st = e / (s * hP), r = e - st * s * hP, k = r / hP, c = r - k * hP;
            const T *cc = D.m2x_c + size_t(k) * nc;
            const cpx<T> *Ms = Mu + st * nc;
            for (int h = 0; h < 2; ++h) {
                const int m = h ? p - c : c;
                if (h && m == c) break;
                T evx = 0, evy = 0, odx = 0, ody = 0;
                for (int n = m; n <= p; n += 2) {
                    const int i = tri(n, m);
                    evx = fma(cc[i], Ms[i].x, evx);
                    evy = fma(cc[i], Ms[i].y, evy);
                }
                for (int n = m + 1; n <= p; n += 2) {
                    const int i = tri(n, m);
                    odx = fma(cc[i], Ms[i].x, odx);
                    ody = fma(cc[i], Ms[i].y, ody);
                }
                const T sg = m == 0 ? T(1) : (((m >> 1) & 1) ? T(-2) : T(2));   // 2 i^m up to i for odd m
                AE[k * NS + m * kSets + st] = mk(sg * evx, sg * evy);
                AO[k * NS + m * kSets + st] = mk(sg * odx, sg * ody);
            }
        }
        __syncthreads();
        if constexpr (sizeof(T) == 8) {
            // W_j = (w_k/M_k) [A^0 + 2 sum_m i^m Re(A^m e^{i m a_j})], A = AE +- AO, all four
            // sets per unit.  Waves t and M_k/2 - t of a node have angles a and pi - a:
            // e^{i m (pi - a)} = (-1)^m conj(e^{i m a}), so with P = sum a.x z.x and
            // Q = sum a.y z.y over even (or odd) m, Re(A z) = P - Q serves wave t and
            // (-1)^m Re(A conj z) = +-(P + Q) its partner: two FMAs per (m, set) for
            // both waves.  Real parts are stored after the even-m pass, imaginary parts
            // after the odd-m pass.
            const size_t dsz = size_t(kSets) * S;
            for (int u = threadIdx.x; u < D.NU; u += blockDim.x) {
                const int k = D.u_k[u];
                const int j0 = D.k_start[k], H = D.k_start[k + 1] - j0, t = u - D.u_start[k], Mk = 2 * H;
                const bool pair = t > 0 && 2 * t != H;
                const int ja = j0 + t, jb = j0 + H - t;
                const cpx<T> *rt = D.roots + 2 * j0;
                const cpx<T> *ae = AE + k * NS;
                const cpx<T> *ao = AO + k * NS;
                const T wm = D.e_wm[ja];
                T pe[kSets], qe[kSets], po[kSets], qo[kSets];
    #pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    pe[st] = ae[st].x;
                    qe[st] = 0;
                    po[st] = ao[st].x;
                    qo[st] = 0;
                }
                int step2 = 2 * t;
                if (step2 >= Mk) step2 -= Mk;
                int idx = 0;   // (m t) mod Mk for even m
                for (int m = 2; m <= p; m += 2) {
                    idx += step2;
                    if (idx >= Mk) idx -= Mk;
                    const cpx<T> z = rt[idx];
    #pragma unroll
                    for (int st = 0; st < kSets; ++st) {
                        const cpx<T> a = ae[m * kSets + st], o = ao[m * kSets + st];
                        pe[st] = fma(a.x, z.x, pe[st]);
                        qe[st] = fma(a.y, z.y, qe[st]);
                        po[st] = fma(o.x, z.x, po[st]);
                        qo[st] = fma(o.y, z.y, qo[st]);
                    }
                }
                // real parts: even m; + direction A = AE + AO, - direction AE - AO
    #pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    const T ea = pe[st] - qe[st], oa = po[st] - qo[st];
                    Xo[base + size_t(2 * (f - f0)) * dsz + st * S + ja].x = wm * (ea + oa);
                    Xo[base + size_t(2 * (f - f0) + 1) * dsz + st * S + ja].x = wm * (ea - oa);
                    if (pair) {
                        const T eb = pe[st] + qe[st], ob = po[st] + qo[st];
                        Xo[base + size_t(2 * (f - f0)) * dsz + st * S + jb].x = wm * (eb + ob);
                        Xo[base + size_t(2 * (f - f0) + 1) * dsz + st * S + jb].x = wm * (eb - ob);
                    }
                    pe[st] = 0;
                    qe[st] = 0;
                    po[st] = 0;
                    qo[st] = 0;
                }
                idx = t;      // odd m, starting at m = 1
                for (int m = 1; m <= p; m += 2) {
                    const cpx<T> z = rt[idx];
    #pragma unroll
                    for (int st = 0; st < kSets; ++st) {
                        const cpx<T> a = ae[m * kSets + st], o = ao[m * kSets + st];
                        pe[st] = fma(a.x, z.x, pe[st]);
                        qe[st] = fma(a.y, z.y, qe[st]);
                        po[st] = fma(o.x, z.x, po[st]);
                        qo[st] = fma(o.y, z.y, qo[st]);
                    }
                    idx += step2;
                    if (idx >= Mk) idx -= Mk;
                }
                // imaginary parts: odd m, the partner with sign (-1)^m = -1
    #pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    const T ea = pe[st] - qe[st], oa = po[st] - qo[st];
                    Xo[base + size_t(2 * (f - f0)) * dsz + st * S + ja].y = wm * (ea + oa);
                    Xo[base + size_t(2 * (f - f0) + 1) * dsz + st * S + ja].y = wm * (ea - oa);
                    if (pair) {
                        const T eb = -(pe[st] + qe[st]), ob = -(po[st] + qo[st]);
                        Xo[base + size_t(2 * (f - f0)) * dsz + st * S + jb].y = wm * (eb + ob);
                        Xo[base + size_t(2 * (f - f0) + 1) * dsz + st * S + jb].y = wm * (eb - ob);
                    }
                }
            }
        } else {
            // FP32: one wave per thread (the kernel is not bound by its FMAs, and
            // twice the threads hide more latency)
            // W_j = (w_k/M_k) [A^0 + 2 sum_m i^m Re(A^m e^{i m a_j})], A = AE +- AO, all four
            // sets per wave (one root lookup and index update serve four sets)
            for (int j = threadIdx.x; j < S; j += blockDim.x) {
                const int k = D.e_k[j];
                const int j0 = D.k_start[k], jl = j - j0, Mk = 2 * (D.k_start[k + 1] - j0);
                const cpx<T> *rt = D.roots + 2 * j0;
                const cpx<T> *ae = AE + k * NS;
                const cpx<T> *ao = AO + k * NS;
                T er[kSets], orr[kSets], ei[kSets], oi[kSets];
    #pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    er[st] = ae[st].x;
                    orr[st] = ao[st].x;
                    ei[st] = 0;
                    oi[st] = 0;
                }
                int step2 = 2 * jl;
                if (step2 >= Mk) step2 -= Mk;
                int idx = 0;   // (m jl) mod Mk for even m
                for (int m = 2; m <= p; m += 2) {
                    idx += step2;
                    if (idx >= Mk) idx -= Mk;
                    const cpx<T> z = rt[idx];
    #pragma unroll
                    for (int st = 0; st < kSets; ++st) {
                        const cpx<T> a = ae[m * kSets + st], o = ao[m * kSets + st];
                        er[st] = fma(-a.y, z.y, fma(a.x, z.x, er[st]));
                        orr[st] = fma(-o.y, z.y, fma(o.x, z.x, orr[st]));
                    }
                }
                idx = jl;      // odd m, starting at m = 1
                for (int m = 1; m <= p; m += 2) {
                    const cpx<T> z = rt[idx];
    #pragma unroll
                    for (int st = 0; st < kSets; ++st) {
                        const cpx<T> a = ae[m * kSets + st], o = ao[m * kSets + st];
                        ei[st] = fma(-a.y, z.y, fma(a.x, z.x, ei[st]));
                        oi[st] = fma(-o.y, z.y, fma(o.x, z.x, oi[st]));
                    }
                    idx += step2;
                    if (idx >= Mk) idx -= Mk;
                }
                const T wm = D.e_wm[j];
    #pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    Xo[base + size_t(2 * (f - f0)) * kSets * S + st * S + j] =
                        mk(wm * (er[st] + orr[st]), wm * (ei[st] + oi[st]));
                    Xo[base + size_t(2 * (f - f0) + 1) * kSets * S + st * S + j] =
                        mk(wm * (er[st] - orr[st]), wm * (ei[st] - oi[st]));
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- X2X merge-and-shift
template <typename T, bool FAC>
__global__ void k_x2x(const int *parents, DevTables<T> D, const int *coll, const int *child, const int *leaf,
                      const cpx<T> *Xo, cpx<T> *Xi, int f0, int nf) {
    __shared__ int src[216];
    __shared__ int vsrc[216], vsh[216], vpre[217];   // the present sources, compacted in slot order
    __shared__ int vend[216];   // child mask of its group at the last present source of a group, else 0
    // FAC (FP32, few plane waves): the shift of a source as the product of its
    // per-axis factors, from shared memory (z offsets x S, x offsets, y offsets);
    // otherwise the shift table
    __shared__ int voz[216], vox[216], voy[216];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int P = parents[blockIdx.x];
    const int dl = blockIdx.y, d = 2 * f0 + dl;   // direction, and its slot in this pass's buffers
    const int S = D.S;
    for (int sl = threadIdx.x; sl < 216; sl += blockDim.x) {
        int q = sl >> 3, o = sl & 7;
        int Q = coll[27 * P + q];
        src[sl] = (Q >= 0 && !leaf[Q]) ? child[8 * Q + o] : -1;
    }
    __syncthreads();
    int ng = D.grp_n[d];
    const int *goff = D.grp_off + d * (kGroupMax + 1);
    const int *gmask = D.grp_mask + d * kGroupMax;
    const int *slots = D.slot_list + d * 216;
    // warp 0: keep the slots whose source box exists; vpre[z] = present slots before z,
    // so group g covers vsrc[vpre[goff[g]] .. vpre[goff[g + 1]])
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, nsl = goff[ng];
        int carry = 0;
        for (int z0 = 0; z0 < nsl; z0 += 32) {
            const int z = z0 + lane;
            int ent = 0, sb = -1;
            if (z < nsl) {
                ent = slots[z];
                sb = src[ent & 255];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, sb >= 0);
            const int pos = carry + __popc(bal & ((1u << lane) - 1u));
            if (z < nsl) vpre[z] = pos;
            if (sb >= 0) {
                vsrc[pos] = sb;
                vsh[pos] = ent >> 8;
            }
            carry += __popc(bal);
        }
        if (lane == 0) vpre[nsl] = carry;
    }
    __syncthreads();
    const int nz = vpre[goff[ng]];
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
        vend[z] = 0;
        const int o = vsh[z];
        vox[z] = (o % 6) * S;
        voy[z] = ((o / 6) % 6) * S;
        voz[z] = (o / 36) * S;
    }
    T *sZ = reinterpret_cast<T *>(smem_raw);
    cpx<T> *sX = reinterpret_cast<cpx<T> *>(sZ + ((6 * S + 3) & ~3));
    cpx<T> *sY = sX + 6 * S;
    if constexpr (FAC) {
        for (int i = threadIdx.x; i < 6 * S; i += blockDim.x) {
            sZ[i] = D.shz[i];
            sX[i] = D.shx[i];
            sY[i] = D.shy[i];
        }
    }
    __syncthreads();
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int z1 = vpre[goff[g + 1]];
        if (z1 > vpre[goff[g]]) vend[z1 - 1] = gmask[g];
    }
    __syncthreads();
    int ch[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) ch[t] = child[8 * P + t];
    const size_t dstride = size_t(2 * nf) * kSets * S;
    const cpx<T> *Xd = Xo + size_t(dl) * kSets * S;
    for (int e = threadIdx.x; e < kSets * S; e += blockDim.x) {
        int j = e % S;
        cpx<T> acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = mk<T>(0, 0);
        // one pass over all present sources (group boundaries marked by vend), so
        // that the unrolled loads run ahead across groups (measured: 8 in flight for the
        // FP32 table form, 4 elsewhere)
        constexpr int kUnroll = (sizeof(T) == 4 && !FAC) ? 8 : 4;
        cpx<T> ga = mk<T>(0, 0);
#pragma unroll kUnroll
        for (int z = 0; z < nz; ++z) {
            const cpx<T> x = Xd[size_t(vsrc[z]) * dstride + e];
            cpx<T> sh;
            if constexpr (FAC) {
                const cpx<T> a = sX[vox[z] + j], b = sY[voy[z] + j];
                const T c = sZ[voz[z] + j];
                sh = mk(c * fmaf(a.x, b.x, -a.y * b.y), c * fmaf(a.x, b.y, a.y * b.x));
            } else {
                sh = D.shift[size_t(vsh[z]) * S + j];
            }
            ga.x = fma(-x.y, sh.y, fma(x.x, sh.x, ga.x));
            ga.y = fma(x.y, sh.x, fma(x.x, sh.y, ga.y));
            const int mask = vend[z];   // block-uniform
            if (mask) {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if ((mask >> t) & 1) acc[t] += ga;
                ga = mk<T>(0, 0);
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (ch[t] < 0) continue;
            cpx<T> sh = D.shift[size_t(D.child_shift[d * 8 + t]) * S + j];
            Xi[(size_t(ch[t]) * (2 * nf) + dl) * kSets * S + e] = acc[t] * sh;
        }
    }
}

// Merge-and-shift with the four charge sets of a plane wave in one thread (the
// FP32 form, and the box-origin form in either precision).  With rb (box origin
// of q4 = F . (r - o)), set 4 travels with its origin at the centre of the box
// whose expansion it is: each source's set 4 moves to the parent centre as it is
// merged, X4 += (c_source - c_parent) . X_F, and each merged sum moves to the
// child as it is shifted there, X4 += (c_parent - c_child) . X_F, with X_F the
// force sets 1..3 of the same wave (rotations of the frames act on the plane-wave
// variables only, so the world offsets apply as they are).
template <typename T, bool FAC>
__global__ void k_x2x4(const int *parents, DevTables<T> D, const int *coll, const int *child, const int *leaf,
                       const double *side, const cpx<T> *Xo, cpx<T> *Xi, int f0, int nf, int rb) {
    __shared__ int src[216];
    __shared__ int vsrc[216], vsh[216], vpre[217], vend[216];
    __shared__ int voz[216], vox[216], voy[216];
    __shared__ T vd[3][216];   // source centre - parent centre (world axes), set-4 origin move
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = parents[blockIdx.x];
    const int dl = blockIdx.y, d = 2 * f0 + dl;
    const int S = D.S;
    const double hc = 0.5 * side[P];   // side of P's children (and of the sources)
    for (int sl = threadIdx.x; sl < 216; sl += blockDim.x) {
        int q = sl >> 3, o = sl & 7;
        int Q = coll[27 * P + q];
        src[sl] = (Q >= 0 && !leaf[Q]) ? child[8 * Q + o] : -1;
    }
    __syncthreads();
    const int ng = D.grp_n[d];
    const int *goff = D.grp_off + d * (kGroupMax + 1);
    const int *gmask = D.grp_mask + d * kGroupMax;
    const int *slots = D.slot_list + d * 216;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, nsl = goff[ng];
        int carry = 0;
        for (int z0 = 0; z0 < nsl; z0 += 32) {
            const int z = z0 + lane;
            int ent = 0, sb = -1;
            if (z < nsl) {
                ent = slots[z];
                sb = src[ent & 255];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, sb >= 0);
            const int pos = carry + __popc(bal & ((1u << lane) - 1u));
            if (z < nsl) vpre[z] = pos;
            if (sb >= 0) {
                vsrc[pos] = sb;
                vsh[pos] = ent >> 8;
                // slot = colleague (dx, dy, dz in -1..1, index 9 dz + 3 dy + dx + 13) x 8 + child octant:
                // source centre - P's centre = hc (2 d + bit - 1/2) per axis, in world axes
                const int sl = ent & 255, q = sl >> 3, o = sl & 7;
                vd[0][pos] = T(hc * (2 * (q % 3 - 1) + (o & 1) - 0.5));
                vd[1][pos] = T(hc * (2 * ((q / 3) % 3 - 1) + ((o >> 1) & 1) - 0.5));
                vd[2][pos] = T(hc * (2 * (q / 9 - 1) + ((o >> 2) & 1) - 0.5));
            }
            carry += __popc(bal);
        }
        if (lane == 0) vpre[nsl] = carry;
    }
    __syncthreads();
    const int nz = vpre[goff[ng]];
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
        vend[z] = 0;
        const int o = vsh[z];
        vox[z] = (o % 6) * S;
        voy[z] = ((o / 6) % 6) * S;
        voz[z] = (o / 36) * S;
    }
    T *sZ = reinterpret_cast<T *>(smem_raw);
    cpx<T> *sX = reinterpret_cast<cpx<T> *>(sZ + ((6 * S + 3) & ~3));
    cpx<T> *sY = sX + 6 * S;
    if constexpr (FAC) {
        for (int i = threadIdx.x; i < 6 * S; i += blockDim.x) {
            sZ[i] = D.shz[i];
            sX[i] = D.shx[i];
            sY[i] = D.shy[i];
        }
    }
    __syncthreads();
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int z1 = vpre[goff[g + 1]];
        if (z1 > vpre[goff[g]]) vend[z1 - 1] = gmask[g];
    }
    __syncthreads();
    int ch[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) ch[t] = child[8 * P + t];
    const size_t dstride = size_t(2 * nf) * kSets * S;
    const cpx<T> *Xd = Xo + size_t(dl) * kSets * S;
    for (int j = threadIdx.x; j < S; j += blockDim.x) {
        cpx<T> acc[8][kSets];
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int k = 0; k < kSets; ++k) acc[t][k] = mk<T>(0, 0);
        cpx<T> ga[kSets];
#pragma unroll
        for (int k = 0; k < kSets; ++k) ga[k] = mk<T>(0, 0);
#pragma unroll 2
        for (int z = 0; z < nz; ++z) {
            const cpx<T> *xs = Xd + size_t(vsrc[z]) * dstride + j;
            cpx<T> x[kSets];
#pragma unroll
            for (int k = 0; k < kSets; ++k) x[k] = xs[size_t(k) * S];
            if (rb) {
                const T ex = vd[0][z], ey = vd[1][z], ez = vd[2][z];
                x[3].x = fma(ez, x[2].x, fma(ey, x[1].x, fma(ex, x[0].x, x[3].x)));
                x[3].y = fma(ez, x[2].y, fma(ey, x[1].y, fma(ex, x[0].y, x[3].y)));
            }
            cpx<T> sh;
            if constexpr (FAC) {
                const cpx<T> a = sX[vox[z] + j], b = sY[voy[z] + j];
                const T c = sZ[voz[z] + j];
                sh = mk(c * fma(a.x, b.x, -a.y * b.y), c * fma(a.x, b.y, a.y * b.x));
            } else {
                sh = D.shift[size_t(vsh[z]) * S + j];
            }
#pragma unroll
            for (int k = 0; k < kSets; ++k) {
                ga[k].x = fma(-x[k].y, sh.y, fma(x[k].x, sh.x, ga[k].x));
                ga[k].y = fma(x[k].y, sh.x, fma(x[k].x, sh.y, ga[k].y));
            }
            const int mask = vend[z];   // block-uniform
            if (mask) {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if ((mask >> t) & 1)
#pragma unroll
                        for (int k = 0; k < kSets; ++k) acc[t][k] += ga[k];
#pragma unroll
                for (int k = 0; k < kSets; ++k) ga[k] = mk<T>(0, 0);
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (ch[t] < 0) continue;
            if (rb) {   // P's centre - child t's centre = -(hc / 2) (2 bit - 1) per axis
                const double h = 0.5 * hc;
                const T ex = T((t & 1) ? -h : h), ey = T((t & 2) ? -h : h), ez = T((t & 4) ? -h : h);
                acc[t][3].x = fma(ez, acc[t][2].x, fma(ey, acc[t][1].x, fma(ex, acc[t][0].x, acc[t][3].x)));
                acc[t][3].y = fma(ez, acc[t][2].y, fma(ey, acc[t][1].y, fma(ex, acc[t][0].y, acc[t][3].y)));
            }
            const cpx<T> sh = D.shift[size_t(D.child_shift[d * 8 + t]) * S + j];
            cpx<T> *dst = Xi + (size_t(ch[t]) * (2 * nf) + dl) * kSets * S + j;
#pragma unroll
            for (int k = 0; k < kSets; ++k) dst[size_t(k) * S] = acc[t][k] * sh;
        }
    }
}

// ---------------------------------------------------------------- bulk copies and mbarriers
// One-dimensional bulk copies global -> shared (the TMA engine) completing on an
// mbarrier: a thread announces the bytes to arrive (expect_tx), issues the copies,
// and every thread waits for the barrier's phase.  Waits give up after about a
// second (a copy that never lands), so that no kernel can hang the device.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return unsigned(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t limit_ns = 1000000000ull) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// Self-test of the bounded wait: one thread waits for an mbarrier phase that no
// arrival will ever complete (no copy is issued), gives up after limit_ns and
// reports the timeout through the status word, as the pipelined kernels do.
__global__ void k_wait_selftest(uint64_t limit_ns, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_init_fence();
    if (!mbar_wait(&bar, 0, limit_ns)) atomicOr(status, DEVERR_TIMEOUT);
}

int wait_selftest(double limit_ms, cudaStream_t st) {
    unsigned *d = nullptr;
    RPY_CHECK(cudaMalloc(&d, sizeof(unsigned)));
    unsigned h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, st>>>(uint64_t(limit_ms * 1e6), d);
        RPY_LAUNCHED(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return check_cuda("wait self-test", e);
    return (h & DEVERR_TIMEOUT) ? RPY_ERR_TIMEOUT : RPY_OK;
}
// orders this thread's earlier generic-proxy accesses to shared memory before later bulk copies
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bulk-copy pipeline of the FP32 X2X: kX2XStages buffers, each holding one source's
// outgoing waves in one direction (4 S values) and its shift row (S values, rows
// padded to an even length).
constexpr int kX2XStages = 4;
__host__ __device__ inline int x2x_tma_stage_elems(int S) { return 4 * S + ((S + 1) & ~1); }
__host__ inline size_t x2x_tma_smem(int S) { return sizeof(cpx<float>) * size_t(kX2XStages) * x2x_tma_stage_elems(S); }

// FP32 merge-and-shift, one consumer thread per plane wave (the four charge sets
// and the box-origin move of set 4 as in k_x2x4), fed by a producer warp: the
// present sources are staged through shared memory by bulk copies (TMA) into
// kX2XStages buffers.  Buffer q is "full" when its copies have landed (an mbarrier
// with the transaction count) and "empty" when every consumer warp has read it
// (an mbarrier with one arrival per consumer warp); the producer refills a buffer
// as soon as it is empty, so the consumers never wait on a global load and the
// block needs no barrier per source.
__global__ void __launch_bounds__(512, 1) k_x2x_tma(const int *parents, DevTables<float> D, const int *coll,
                                                    const int *child, const int *leaf, const double *side,
                                                    const cpx<float> *Xo, cpx<float> *Xi, int f0, int nf, int rb,
                                                    unsigned *status) {
    __shared__ int src[216];
    __shared__ int vsrc[216], vsh[216], vpre[217], vend[216];
    __shared__ float vd[3][216];
    __shared__ __align__(8) uint64_t full[kX2XStages], empty[kX2XStages];
    __shared__ int bad, issued;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = parents[blockIdx.x];
    const int dl = blockIdx.y, d = 2 * f0 + dl;
    const int S = D.S, Sp = D.Sp;
    const int ncw = (S + 31) / 32;                 // consumer warps; the last warp produces
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double hc = 0.5 * side[P];
    for (int sl = threadIdx.x; sl < 216; sl += blockDim.x) {
        int q = sl >> 3, o = sl & 7;
        int Q = coll[27 * P + q];
        src[sl] = (Q >= 0 && !leaf[Q]) ? child[8 * Q + o] : -1;
    }
    if (threadIdx.x == 0) {
        bad = 0;
        issued = 0;
        for (int q = 0; q < kX2XStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], unsigned(ncw));
        }
        mbar_init_fence();
    }
    __syncthreads();
    const int ng = D.grp_n[d];
    const int *goff = D.grp_off + d * (kGroupMax + 1);
    const int *gmask = D.grp_mask + d * kGroupMax;
    const int *slots = D.slot_list + d * 216;
    if (warp == 0) {
        const int nsl = goff[ng];
        int carry = 0;
        for (int z0 = 0; z0 < nsl; z0 += 32) {
            const int z = z0 + lane;
            int ent = 0, sb = -1;
            if (z < nsl) {
                ent = slots[z];
                sb = src[ent & 255];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, sb >= 0);
            const int pos = carry + __popc(bal & ((1u << lane) - 1u));
            if (z < nsl) vpre[z] = pos;
            if (sb >= 0) {
                vsrc[pos] = sb;
                vsh[pos] = ent >> 8;
                const int sl = ent & 255, q = sl >> 3, o = sl & 7;
                vd[0][pos] = float(hc * (2 * (q % 3 - 1) + (o & 1) - 0.5));
                vd[1][pos] = float(hc * (2 * ((q / 3) % 3 - 1) + ((o >> 1) & 1) - 0.5));
                vd[2][pos] = float(hc * (2 * (q / 9 - 1) + ((o >> 2) & 1) - 0.5));
            }
            carry += __popc(bal);
        }
        if (lane == 0) vpre[nsl] = carry;
    }
    __syncthreads();
    const int nz = vpre[goff[ng]];
    for (int z = threadIdx.x; z < nz; z += blockDim.x) vend[z] = 0;
    __syncthreads();
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int z1 = vpre[goff[g + 1]];
        if (z1 > vpre[goff[g]]) vend[z1 - 1] = gmask[g];
    }
    __syncthreads();
    const int stage_elems = x2x_tma_stage_elems(S);
    cpx<float> *stage0 = reinterpret_cast<cpx<float> *>(smem_raw);
    if (warp == ncw) {
        // producer: one lane issues the copies, refilling each buffer once it is empty
        if (lane == 0) {
            const size_t dstride = size_t(2 * nf) * kSets * S;
            const cpx<float> *Xd = Xo + size_t(dl) * kSets * S;
            const unsigned src_bytes = 32u * unsigned(S), sh_bytes = 8u * unsigned(Sp);
            for (int z = 0; z < nz; ++z) {
                const int q = z % kX2XStages;
                if (z >= kX2XStages && !mbar_wait(&empty[q], unsigned(z / kX2XStages - 1) & 1u)) {
                    bad = 1;
                    break;
                }
                if (*(volatile int *)&bad) break;
                cpx<float> *buf = stage0 + size_t(q) * stage_elems;
                mbar_expect(&full[q], src_bytes + sh_bytes);
                bulk_load(buf, Xd + size_t(vsrc[z]) * dstride, src_bytes, &full[q]);
                bulk_load(buf + 4 * S, D.shiftp + size_t(vsh[z]) * Sp, sh_bytes, &full[q]);
                issued = z + 1;
            }
        }
    } else {
        int ch[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) ch[t] = child[8 * P + t];
        const int j = threadIdx.x;
        const bool act = j < S;
        cpx<float> acc[8][kSets];
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int k = 0; k < kSets; ++k) acc[t][k] = mk(0.f, 0.f);
        cpx<float> ga[kSets];
#pragma unroll
        for (int k = 0; k < kSets; ++k) ga[k] = mk(0.f, 0.f);
        for (int z = 0; z < nz; ++z) {
            const int q = z % kX2XStages;
            if (!mbar_wait(&full[q], unsigned(z / kX2XStages) & 1u) || *(volatile int *)&bad) {
                bad = 1;
                break;
            }
            if (act) {
                const cpx<float> *buf = stage0 + size_t(q) * stage_elems;
                cpx<float> x[kSets];
#pragma unroll
                for (int k = 0; k < kSets; ++k) x[k] = buf[k * S + j];
                if (rb) {
                    const float ex = vd[0][z], ey = vd[1][z], ez = vd[2][z];
                    x[3].x = fmaf(ez, x[2].x, fmaf(ey, x[1].x, fmaf(ex, x[0].x, x[3].x)));
                    x[3].y = fmaf(ez, x[2].y, fmaf(ey, x[1].y, fmaf(ex, x[0].y, x[3].y)));
                }
                const cpx<float> sh = buf[4 * S + j];
#pragma unroll
                for (int k = 0; k < kSets; ++k) {
                    ga[k].x = fmaf(-x[k].y, sh.y, fmaf(x[k].x, sh.x, ga[k].x));
                    ga[k].y = fmaf(x[k].y, sh.x, fmaf(x[k].x, sh.y, ga[k].y));
                }
                const int mask = vend[z];   // block-uniform
                if (mask) {
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if ((mask >> t) & 1)
#pragma unroll
                            for (int k = 0; k < kSets; ++k) acc[t][k] += ga[k];
#pragma unroll
                    for (int k = 0; k < kSets; ++k) ga[k] = mk(0.f, 0.f);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[q]);   // this warp is done with buffer q
        }
        if (!*(volatile int *)&bad && act) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (ch[t] < 0) continue;
                if (rb) {   // P's centre - child t's centre = -(hc / 2) (2 bit - 1) per axis
                    const float h = float(0.5 * hc);
                    const float ex = (t & 1) ? -h : h, ey = (t & 2) ? -h : h, ez = (t & 4) ? -h : h;
                    acc[t][3].x = fmaf(ez, acc[t][2].x, fmaf(ey, acc[t][1].x, fmaf(ex, acc[t][0].x, acc[t][3].x)));
                    acc[t][3].y = fmaf(ez, acc[t][2].y, fmaf(ey, acc[t][1].y, fmaf(ex, acc[t][0].y, acc[t][3].y)));
                }
                const cpx<float> sh = D.shift[size_t(D.child_shift[d * 8 + t]) * S + j];
                cpx<float> *dst = Xi + (size_t(ch[t]) * (2 * nf) + dl) * kSets * S + j;
#pragma unroll
                for (int k = 0; k < kSets; ++k) dst[size_t(k) * S] = acc[t][k] * sh;
            }
        }
    }
    __syncthreads();
    if (bad && threadIdx.x == 0) {
        // a wait gave up: let every copy issued land (bounded) before the block's shared
        // memory is released, and flag the failure
        for (int q = 0; q < min(issued, kX2XStages); ++q) {
            const int zl = q + ((issued - 1 - q) / kX2XStages) * kX2XStages;   // last copy issued into buffer q
            mbar_wait(&full[q], unsigned(zl / kX2XStages) & 1u);
        }
        atomicOr(status, DEVERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------- X2L
template <typename T>
__global__ void k_x2l(int b0, int nb, DevTables<T> D, const cpx<T> *Xi, cpx<T> *L, int f0, int nf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = b0 + blockIdx.x;
    const int p = D.p, nc = ncoef(p), s = D.s, S = D.S, P1 = p + 1;
    const int NU = D.NU;
    // per wave-pair unit u (waves t and M_k/2 - t of node k; see k_m2x), one set:
    // Re and Im of I_t +- I_partner for the + direction (UQ[0..3]) and the - direction (UQ[4..7])
    T *UQ = reinterpret_cast<T *>(smem_raw);
    cpx<T> *Bp = reinterpret_cast<cpx<T> *>(UQ + 8 * NU);  // [s][P1]
    cpx<T> *Bm = Bp + s * P1;
    cpx<T> *Lf = Bm + s * P1;                             // [4][nc] frame accumulation
    cpx<T> *Lw = Lf + kSets * nc;                         // [4][nc] world accumulation
    cpx<T> *Lr = Lw + kSets * nc;                         // [4][nc] rotated
    cpx<T> *Tm = Lr + kSets * nc;                         // [4][nc] rotation scratch
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] = mk<T>(0, 0);
    for (int f = f0; f < f0 + nf; ++f) {
        for (int st = 0; st < kSets; ++st) {
            __syncthreads();
            const cpx<T> *sp = Xi + ((size_t(b) * (2 * nf) + 2 * (f - f0)) * kSets + st) * S;
            const cpx<T> *sm = Xi + ((size_t(b) * (2 * nf) + 2 * (f - f0) + 1) * kSets + st) * S;
            for (int u = threadIdx.x; u < NU; u += blockDim.x) {
                const int k = D.u_k[u], j0 = D.k_start[k], H = D.k_start[k + 1] - j0, t = u - D.u_start[k];
                const bool pair = t > 0 && 2 * t != H;
                const cpx<T> pa = sp[j0 + t], ma = sm[j0 + t];
                const cpx<T> pb = pair ? sp[j0 + H - t] : mk<T>(0, 0), mb = pair ? sm[j0 + H - t] : mk<T>(0, 0);
                UQ[u] = pa.x + pb.x;
                UQ[NU + u] = pa.x - pb.x;
                UQ[2 * NU + u] = pa.y + pb.y;
                UQ[3 * NU + u] = pa.y - pb.y;
                UQ[4 * NU + u] = ma.x + mb.x;
                UQ[5 * NU + u] = ma.x - mb.x;
                UQ[6 * NU + u] = ma.y + mb.y;
                UQ[7 * NU + u] = ma.y - mb.y;
            }
            __syncthreads();
            // b_k^m = sum_{j < M_k/2} (I_j + (-1)^m conj I_j) e^{-i m a_j}
            //       = 2 sum_j Re(I_j) e^{-i m a_j}      (m even)
            //       = 2i sum_j Im(I_j) e^{-i m a_j}     (m odd; the factor i is applied below)
            // With e^{-i m (pi - a)} = (-1)^m conj(e^{-i m a}), a wave pair adds
            // (v + (-1)^m v') cos(m a) - i (v - (-1)^m v') sin(m a): even m take the
            // sum and difference of the real parts, odd m those of the imaginary parts.
            for (int e = threadIdx.x; e < s * P1; e += blockDim.x) {
                const int k = e / P1, m = e - k * P1;
                const int j0 = D.k_start[k], Mk = 2 * (D.k_start[k + 1] - j0);
                const int u0 = D.u_start[k], u1 = D.u_start[k + 1];
                const int mm = m % Mk;
                const cpx<T> *rt = D.roots + 2 * j0;
                const T *xp = UQ + ((m & 1) ? 3 : 0) * NU, *yp = UQ + ((m & 1) ? 2 : 1) * NU;
                const T *xm = xp + 4 * NU, *ym = yp + 4 * NU;
                T bpx = 0, bpy = 0, bmx = 0, bmy = 0;
                int idx = 0;
                for (int u = u0; u < u1; ++u) {
                    const cpx<T> r = rt[idx];
                    bpx = fma(xp[u], r.x, bpx);
                    bpy = fma(-yp[u], r.y, bpy);
                    bmx = fma(xm[u], r.x, bmx);
                    bmy = fma(-ym[u], r.y, bmy);
                    idx += mm;
                    if (idx >= Mk) idx -= Mk;
                }
                // the + direction and the reflected - direction enter L through
                // b+ + b- (n + m even) and b+ - b- (n + m odd)
                Bp[e] = mk(bpx + bmx, bpy + bmy);
                Bm[e] = mk(bpx - bmx, bpy - bmy);
            }
            __syncthreads();
            // L_n^m = i^m sum_k (-lambda_k)^n / sqrt((n-m)!(n+m)!) b_k^m, the - direction reflected
            for (int i = threadIdx.x; i < nc; i += blockDim.x) {
                int n = deg_of(i), m = i - tri(n, 0);
                const cpx<T> *Bs = ((n + m) & 1) ? Bm : Bp;
                cpx<T> a = mk<T>(0, 0);
                for (int k = 0; k < s; ++k) {
                    T c = D.x2l_c[size_t(k) * nc + i];
                    cpx<T> bb = Bs[k * P1 + m];
                    a.x = fma(c, bb.x, a.x);
                    a.y = fma(c, bb.y, a.y);
                }
                Lf[st * nc + i] = mul_ipow(mk(2 * a.x, 2 * a.y), m + (m & 1));
            }
        }
        __syncthreads();
        if (f == 0) {
            for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] += Lf[i];
        } else {
            rotate_sets_f<T, true>(D.frot_bwd + size_t(f - 1) * D.frot_len, D.frot_off, p, Lf, Tm, Lr);
            __syncthreads();
            for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] += Lr[i];
        }
    }
    __syncthreads();
    cpx<T> *dst = L + size_t(b) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) dst[i] += Lw[i];
}

// FP32 form of X2L: the four charge sets in one pass.  The incoming waves of a
// frame are staged planar (real parts of the four sets in one float4, imaginary
// parts in another), so that the real DFT, which takes the real parts for even m
// and the imaginary parts for odd m, reads four sets with one 16-byte load per
// wave and direction; one root lookup then serves sixteen FMAs.
__global__ void k_x2l4(int b0, int nb, DevTables<float> D, const cpx<float> *Xi, cpx<float> *L, int f0, int nf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = b0 + blockIdx.x;
    const int p = D.p, nc = ncoef(p), s = D.s, S = D.S, P1 = p + 1;
    float4 *PRe = reinterpret_cast<float4 *>(smem_raw);   // [S] + direction, real parts of sets 0..3
    float4 *PIm = PRe + S;
    float4 *MRe = PIm + S;                                  // - direction
    float4 *MIm = MRe + S;
    // b+ + b- (Bs) and b+ - b- (Bd) per (node, m), as planes of set pairs: (re, im) of sets
    // 0 and 1, then of sets 2 and 3, so that each thread's 16-byte stores are contiguous
    // across lanes (one [s][P1][4] array took four 8-byte stores 32 bytes apart)
    const int SP = s * P1;
    float4 *Bs01 = MIm + S, *Bs23 = Bs01 + SP, *Bd01 = Bs23 + SP, *Bd23 = Bd01 + SP;
    cpx<float> *Lf = reinterpret_cast<cpx<float> *>(Bd23 + SP);                  // [4][nc]
    cpx<float> *Lw = Lf + kSets * nc;
    cpx<float> *Lr = Lw + kSets * nc;
    cpx<float> *Tm = Lr + kSets * nc;                             // rotation scratch
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] = mk<float>(0, 0);
    for (int f = f0; f < f0 + nf; ++f) {
        __syncthreads();
        const cpx<float> *sp = Xi + (size_t(b) * (2 * nf) + 2 * (f - f0)) * kSets * S;
        const cpx<float> *sm = Xi + (size_t(b) * (2 * nf) + 2 * (f - f0) + 1) * kSets * S;
        for (int j = threadIdx.x; j < S; j += blockDim.x) {
            const cpx<float> p0 = sp[j], p1 = sp[S + j], p2 = sp[2 * S + j], p3 = sp[3 * S + j];
            const cpx<float> m0 = sm[j], m1 = sm[S + j], m2 = sm[2 * S + j], m3 = sm[3 * S + j];
            PRe[j] = make_float4(p0.x, p1.x, p2.x, p3.x);
            PIm[j] = make_float4(p0.y, p1.y, p2.y, p3.y);
            MRe[j] = make_float4(m0.x, m1.x, m2.x, m3.x);
            MIm[j] = make_float4(m0.y, m1.y, m2.y, m3.y);
        }
        __syncthreads();
        // b_k^m = 2 sum_j Re(I_j) e^{-i m a_j} (m even), 2i sum_j Im(I_j) e^{-i m a_j} (m odd)
        // (node, m) items at a stride of PA = 8 per node when p + 1 <= 8, so that a
        // quarter-warp never straddles two nodes (its wave loads are then broadcasts)
        const int PA = P1 <= 8 ? 8 : P1;
        for (int ea = threadIdx.x; ea < s * PA; ea += blockDim.x) {
            const int k = ea / PA, m = ea - k * PA;
            if (m >= P1) continue;
            const int e = k * P1 + m;
            const int j0 = D.k_start[k], j1 = D.k_start[k + 1];
            const int Mk = 2 * (j1 - j0), mm = m % Mk;
            const cpx<float> *rt = D.roots + 2 * j0;
            const float4 *vp = (m & 1) ? PIm : PRe;
            const float4 *vm = (m & 1) ? MIm : MRe;
            float bpx[kSets] = {0, 0, 0, 0}, bpy[kSets] = {0, 0, 0, 0};
            float bmx[kSets] = {0, 0, 0, 0}, bmy[kSets] = {0, 0, 0, 0};
            int idx = 0;
            for (int j = j0; j < j1; ++j) {
                const cpx<float> r = rt[idx];
                const float4 a = vp[j], c = vm[j];
                const float av[kSets] = {a.x, a.y, a.z, a.w}, cv[kSets] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int st = 0; st < kSets; ++st) {
                    bpx[st] = fmaf(av[st], r.x, bpx[st]);
                    bpy[st] = fmaf(-av[st], r.y, bpy[st]);
                    bmx[st] = fmaf(cv[st], r.x, bmx[st]);
                    bmy[st] = fmaf(-cv[st], r.y, bmy[st]);
                }
                idx += mm;
                if (idx >= Mk) idx -= Mk;
            }
            Bs01[e] = make_float4(bpx[0] + bmx[0], bpy[0] + bmy[0], bpx[1] + bmx[1], bpy[1] + bmy[1]);
            Bs23[e] = make_float4(bpx[2] + bmx[2], bpy[2] + bmy[2], bpx[3] + bmx[3], bpy[3] + bmy[3]);
            Bd01[e] = make_float4(bpx[0] - bmx[0], bpy[0] - bmy[0], bpx[1] - bmx[1], bpy[1] - bmy[1]);
            Bd23[e] = make_float4(bpx[2] - bmx[2], bpy[2] - bmy[2], bpx[3] - bmx[3], bpy[3] - bmy[3]);
        }
        __syncthreads();
        // L_n^m = i^m sum_k (-lambda_k)^n / sqrt((n-m)!(n+m)!) b_k^m, the - direction reflected
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const int n = deg_of(i), m = i - tri(n, 0);
            const bool odd = (n + m) & 1;
            const float4 *B01 = odd ? Bd01 : Bs01, *B23 = odd ? Bd23 : Bs23;
            // sum over the quadrature nodes with compensated (Kahan) addition: the terms
            // (-lambda_k)^n b_k^m alternate in sign and cancel strongly at high degree
            float ax[kSets] = {0, 0, 0, 0}, ay[kSets] = {0, 0, 0, 0};
            float cx[kSets] = {0, 0, 0, 0}, cy[kSets] = {0, 0, 0, 0};
            auto kahan = [](float &sum, float &c, float v) {
                const float y = v - c, t = sum + y;
                c = (t - sum) - y;
                sum = t;
            };
            for (int k = 0; k < s; ++k) {
                const float c = D.x2l_c[size_t(k) * nc + i];
                const float4 b01 = B01[k * P1 + m], b23 = B23[k * P1 + m];
                kahan(ax[0], cx[0], c * b01.x);
                kahan(ay[0], cy[0], c * b01.y);
                kahan(ax[1], cx[1], c * b01.z);
                kahan(ay[1], cy[1], c * b01.w);
                kahan(ax[2], cx[2], c * b23.x);
                kahan(ay[2], cy[2], c * b23.y);
                kahan(ax[3], cx[3], c * b23.z);
                kahan(ay[3], cy[3], c * b23.w);
            }
#pragma unroll
            for (int st = 0; st < kSets; ++st) Lf[st * nc + i] = mul_ipow(mk(2 * ax[st], 2 * ay[st]), m + (m & 1));
        }
        __syncthreads();
        if (f == 0) {
            for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] += Lf[i];
        } else {
            rotate_sets_f<float, false>(D.frot_bwd + size_t(f - 1) * D.frot_len, D.frot_off, p, Lf, Tm, Lr);
            __syncthreads();
            for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) Lw[i] += Lr[i];
        }
    }
    __syncthreads();
    cpx<float> *dst = L + size_t(b) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) dst[i] += Lw[i];
}

static size_t smem_x2l4(int p, int s, int S) {
    const int nc = ncoef(p);
    return sizeof(float4) * 4 * size_t(S) + sizeof(cpx<float>) * (2 * kSets * s * (p + 1) + 4 * kSets * nc);
}

// ---------------------------------------------------------------- far-field evaluation
constexpr int kNE = 18;   // evaluation expansions of Eq. (2.8) per box
constexpr int kNF = 12;   // evaluated per bead after the fold of k_eval_prep (per-potential form)
constexpr int kNF2 = 6;   // evaluated per bead in the one-expansion-per-component form

// Build the 18 evaluation expansions of Eq. (2.8) from 4 source expansions.
// IRREG = multipole source (degrees grow by one per derivative), else local.
template <typename T, bool IRREG>
__device__ void build_eval_set(const cpx<T> *src, int p, int P, cpx<T> *EV, cpx<T> *tmp, double cbx, double cby,
                               double cbz, const Lad<T> &G) {
    const int st = ncoef(P);
    // 0..2 values
    for (int i = threadIdx.x; i < 3 * st; i += blockDim.x) {
        int k = i / st, c = i - k * st;
        EV[k * st + c] = c < ncoef(p) ? src[k * ncoef(p) + c] : mk<T>(0, 0);
    }
    // 3..11 gradients of sets 0..2 (index 3 + 3k + a), tmp[0..2] gradient of set 3
    for (int k = 0; k < 4; ++k) {
        cpx<T> *gx = k < 3 ? EV + (3 + 3 * k) * st : tmp;
        if (IRREG) d_multipole(src + k * ncoef(p), p, gx, gx + st, gx + 2 * st, P, G);
        else d_local(src + k * ncoef(p), p, gx, gx + st, gx + 2 * st, P, G);
    }
    __syncthreads();
    // 12..14: G4'_a = dL4_a - sum_k cb_k dL_k,a ; tmp[3] = L_C = dxL1 + dyL2 + dzL3
    T cb[3] = {T(cbx), T(cby), T(cbz)};
    for (int i = threadIdx.x; i < st; i += blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            cpx<T> g = tmp[a * st + i];
            for (int k = 0; k < 3; ++k) {
                cpx<T> v = EV[(3 + 3 * k + a) * st + i];
                g.x -= cb[k] * v.x;
                g.y -= cb[k] * v.y;
            }
            EV[(12 + a) * st + i] = g;
        }
        cpx<T> lc = EV[(3 + 0) * st + i] + EV[(3 + 3 + 1) * st + i] + EV[(3 + 6 + 2) * st + i];
        tmp[3 * st + i] = lc;
    }
    __syncthreads();
    int pl = IRREG ? p + 1 : p - 1;
    if (IRREG) d_multipole(tmp + 3 * st, pl, EV + 15 * st, EV + 16 * st, EV + 17 * st, P, G);
    else d_local(tmp + 3 * st, pl, EV + 15 * st, EV + 16 * st, EV + 17 * st, P, G);
    __syncthreads();
}

// rb: the multipoles carry q4 about their own box centres (box origin), so the
// set-4 gradient is re-based from the source box's centre to the leaf's.
template <typename T>
__global__ void k_far_eval(const int *leaves, DevTables<T> D, const int *beg, const int *end, const double *ctr,
                           const double *side, const int *lvl, const int *bsys, const int *woff, const int *widx,
                           const double *pos, int64_t n, SysConst sc, const cpx<T> *L, const cpx<T> *M,
                           double *ufar, int rb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int li = blockIdx.x;
    int b = leaves[li];
    const int p = D.p, nc = ncoef(p), P = p + 2, st = ncoef(P);
    T *smr = reinterpret_cast<T *>(smem_raw);
    Rec<T> R = load_rec(D, smr);
    Lad<T> G = load_lad(D, smr + rec_floats<T>(p));
    cpx<T> *EV = reinterpret_cast<cpx<T> *>(smr + tab_floats<T>(p));
    cpx<T> *tmp = EV + kNE * st;
    cpx<T> *srcs = tmp + 4 * st;
    int sy = bsys[b];
    const double C1 = sc.pc[sy].C1, C2 = sc.pc[sy].C2, icube = sc.pc[sy].icube;
    double c0x = sc.cube[4 * sy], c0y = sc.cube[4 * sy + 1], c0z = sc.cube[4 * sy + 2];
    double cbx = ctr[3 * b], cby = ctr[3 * b + 1], cbz = ctr[3 * b + 2];
    int j0 = beg[b], j1 = end[b];
    int nw = woff[li + 1] - woff[li];
    if (nw == 0) return;
    for (int jc = j0; jc < j1; jc += blockDim.x) {
        int j = jc + threadIdx.x;
        bool act = j < j1;
        double x = act ? pos[j] : cbx, y = act ? pos[n + j] : cby, z = act ? pos[2 * n + j] : cbz;
        double u[3] = {0, 0, 0};
        for (int w = 0; w < nw; ++w) {
            int C = w < 0 ? b : widx[woff[li] + w];
            const cpx<T> *E = w < 0 ? L + size_t(C) * kSets * nc : M + size_t(C) * kSets * nc;
            __syncthreads();
            for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) srcs[i] = E[i];
            __syncthreads();
            // origin of the source expansion's q4: its own centre (box origin) or the cube centre
            const double ox = rb ? ctr[3 * C] : c0x, oy = rb ? ctr[3 * C + 1] : c0y, oz = rb ? ctr[3 * C + 2] : c0z;
            if (w < 0) build_eval_set<T, false>(srcs, p, P, EV, tmp, cbx - ox, cby - oy, cbz - oz, G);
            else build_eval_set<T, true>(srcs, p, P, EV, tmp, cbx - ox, cby - oy, cbz - oz, G);
            double ih = icube * pow2i(lvl[C]);   // 1 / side[C], exactly
            T acc[kNE];
#pragma unroll
            for (int q = 0; q < kNE; ++q) acc[q] = 0;
            T vx = T((x - ctr[3 * C]) * ih), vy = T((y - ctr[3 * C + 1]) * ih), vz = T((z - ctr[3 * C + 2]) * ih);
            if (w < 0) eval_fields<T, kNE, false>(vx, vy, vz, p, EV, st, R.a, R.b, R.c, acc);
            else eval_fields<T, kNE, true>(vx, vy, vz, P, EV, st, R.a, R.b, R.c, acc);
            double xi[3] = {(x - cbx) * ih, (y - cby) * ih, (z - cbz) * ih};
            for (int d = 0; d < 3; ++d) {
                double v = double(acc[d]);
                for (int k = 0; k < 3; ++k) v -= xi[k] * double(acc[3 + 3 * k + d]);
                u[d] += C1 * ih * v + C1 * ih * ih * double(acc[12 + d]) - C2 * ih * ih * ih * double(acc[15 + d]);
            }
        }
        if (act)
            for (int d = 0; d < 3; ++d) ufar[3 * size_t(j) + d] += u[d];
    }
}

// Per leaf at level >= 2: the 18 derived local expansions of Eq. (2.8),
// written to global memory for the bead-parallel evaluation.
// rb: the local expansions carry q4 about their own box centres (box origin),
// so set 4 needs no re-basing to the leaf centre.
template <typename T>
__global__ void k_eval_prep(const int *leaves, DevTables<T> D, const double *ctr, const int *lvl, const int *bsys,
                            SysConst sc, const cpx<T> *L, cpx<T> *EVg, int per_component, int rb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int li = blockIdx.x;
    int b = leaves[li];
    if (lvl[b] < 2) return;
    const int p = D.p, nc = ncoef(p);
    T *smr = reinterpret_cast<T *>(smem_raw);
    Lad<T> G = load_lad(D, smr);
    cpx<T> *srcs = reinterpret_cast<cpx<T> *>(smr + ((6 * ncoef(p + 2) + 1) & ~1));
    cpx<T> *tmp = srcs + kSets * nc;
    const cpx<T> *E = L + size_t(b) * kSets * nc;
    for (int i = threadIdx.x; i < kSets * nc; i += blockDim.x) srcs[i] = E[i];
    __syncthreads();
    int sy = bsys[b];
    cpx<T> *EV = EVg + size_t(li) * kNE * nc;
    if (rb) build_eval_set<T, false>(srcs, p, p, EV, tmp, 0.0, 0.0, 0.0, G);
    else
        build_eval_set<T, false>(srcs, p, p, EV, tmp, ctr[3 * b] - sc.cube[4 * sy],
                                 ctr[3 * b + 1] - sc.cube[4 * sy + 1], ctr[3 * b + 2] - sc.cube[4 * sy + 2], G);
    // Fold the terms of Eq. (2.8) that are not multiplied by a coordinate into
    // fields 0..2 (in units of C1/h):  L_d + h^-1 dL4'_d - (C2/C1) h^-2 dL_C,d.
    // The bead evaluation then needs fields 0..11 only.
    const double ih = sc.pc[sy].icube * pow2i(lvl[b]);
    const T c4 = T(ih), cc = T(sc.pc[sy].C2 / sc.pc[sy].C1 * ih * ih);
    for (int i = threadIdx.x; i < 3 * nc; i += blockDim.x) {
        int d = i / nc, c = i - d * nc;
        cpx<T> v = EV[d * nc + c], g4 = EV[(12 + d) * nc + c], gc = EV[(15 + d) * nc + c];
        v.x = fma(c4, g4.x, fma(-cc, gc.x, v.x));
        v.y = fma(c4, g4.y, fma(-cc, gc.y, v.y));
        EV[d * nc + c] = v;
    }
    int nf = kNF;
    if (per_component) {
        // Approach 2 of Sec. 2: one expansion per velocity component.  With
        // G_kd = dL_k/dx_d (fields 3 + 3k + d, degree <= p - 1) and x the bead
        // offset in box units, sum_k x_k G_kd = A_d + |x|^2 B_d with A_d, B_d
        // harmonic: for each degree-n part h of G_kd, with g = h / (2n + 1),
        //   x_k h = [x_k h - |x|^2 d_k g] + |x|^2 d_k g,
        // where the bracket is -|x|^(2n+3) d_k(g / |x|^(2n+1)) (Kelvin transform:
        // the same coefficients read as a multipole expansion), so
        //   A_d = -sum_k [d_k of g as a multipole, read as a local expansion],
        //   B_d =  sum_k [d_k of g as a local expansion].
        // Fields become H_d = F_d - A_d (0..2, degree <= p) and B_d (3..5).
        __syncthreads();
        for (int i = threadIdx.x; i < 9 * nc; i += blockDim.x) {
            const int c = i % nc;
            const T w = T(1) / T(2 * deg_of(c) + 1);
            cpx<T> v = EV[3 * nc + i];
            EV[3 * nc + i] = mk(w * v.x, w * v.y);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * nc; i += blockDim.x) {
            const int d = i / nc, c = i - d * nc;
            cpx<T> a = mk<T>(0, 0), bb = mk<T>(0, 0);
            for (int k = 0; k < 3; ++k) {
                const cpx<T> *g = EV + (3 + 3 * k + d) * nc;
                a += d_mul_one(g, p - 1, k, c, G);
                bb += d_loc_one(g, p - 1, k, c, G);
            }
            EV[d * nc + c] += a;
            EV[(12 + d) * nc + c] = bb;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * nc; i += blockDim.x) EV[3 * nc + i] = EV[12 * nc + i];
        nf = kNF2;
    }
    __syncthreads();
    // the evaluated fields carry the factor 2 of the m > 0 terms of Re(sum E h)
    for (int i = threadIdx.x; i < nf * nc; i += blockDim.x) {
        int c = i % nc, n = deg_of(c);
        if (c != tri(n, 0)) {
            cpx<T> v = EV[i];
            EV[i] = mk(2 * v.x, 2 * v.y);
        }
    }
}

// One thread per bead: L2P of the leaf's derived expansions and Eq. (2.8),
// per potential (NF = 12: folded values and nine gradients) or per velocity
// component (NF = 6: u_d = H_d - |x|^2 B_d).
template <typename T, int NF>
__global__ void k_eval_apply(int64_t n, const int *bead_leaf, const int *leaves, DevTables<T> D, const double *ctr,
                             const double *side, const int *lvl, const int *bsys, const double *pos, SysConst sc,
                             const cpx<T> *EVg, double *ufar) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int li = bead_leaf[i];
    int b = leaves[li];
    double u[3] = {0, 0, 0};
    if (lvl[b] >= 2) {
        const int p = D.p, nc = ncoef(p);
        int sy = bsys[b];
        const double C1 = sc.pc[sy].C1;
        const double ih = sc.pc[sy].icube * pow2i(lvl[b]);   // 1 / side[b], exactly
        double xi[3] = {(pos[i] - ctr[3 * b]) * ih, (pos[n + i] - ctr[3 * b + 1]) * ih,
                        (pos[2 * n + i] - ctr[3 * b + 2]) * ih};
        T acc[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) acc[q] = 0;
        eval_fields<T, NF, false, true>(T(xi[0]), T(xi[1]), T(xi[2]), p, EVg + size_t(li) * kNE * nc, nc, D.rec_a,
                                        D.rec_b, D.rec_c, acc);
        if constexpr (NF == kNF2) {
            // fields 0..2: H_d; 3..5: B_d
            const double r2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
            for (int d = 0; d < 3; ++d) u[d] = C1 * ih * (double(acc[d]) - r2 * double(acc[3 + d]));
        } else {
            // fields 0..2: the folded value terms; 3..11: gradients dL_k / dx_d at 3 + 3k + d
            for (int d = 0; d < 3; ++d) {
                double v = double(acc[d]);
                for (int k = 0; k < 3; ++k) v -= xi[k] * double(acc[3 + 3 * k + d]);
                u[d] = C1 * ih * v;
            }
        }
    }
    for (int d = 0; d < 3; ++d) ufar[3 * i + d] = u[d];
}

// Laplace diagnostic: potential, gradient and Hessian of each set from L2P and M2P.
template <typename T, bool IRREG>
__device__ void build_lap_set(const cpx<T> *src, int p, int P, cpx<T> *EV, cpx<T> *tmp, const Lad<T> &G) {
    const int st = ncoef(P);
    for (int i = threadIdx.x; i < st; i += blockDim.x) EV[i] = i < ncoef(p) ? src[i] : mk<T>(0, 0);
    if (IRREG) d_multipole(src, p, EV + st, EV + 2 * st, EV + 3 * st, P, G);
    else d_local(src, p, EV + st, EV + 2 * st, EV + 3 * st, P, G);
    __syncthreads();
    int pd = IRREG ? p + 1 : p - 1;
    // Hessian rows: d/dx of (x, y, z) derivatives -> 4..6, d/dy -> 7..9, d/dz -> 10..12
    for (int a = 0; a < 3; ++a) {
        if (IRREG) d_multipole(EV + (1 + a) * st, pd, tmp, tmp + st, tmp + 2 * st, P, G);
        else d_local(EV + (1 + a) * st, pd, tmp, tmp + st, tmp + 2 * st, P, G);
        __syncthreads();
        for (int i = threadIdx.x; i < st; i += blockDim.x)
            for (int c = 0; c < 3; ++c) EV[(4 + 3 * a + c) * st + i] = tmp[c * st + i];
        __syncthreads();
    }
}

template <typename T>
__global__ void k_lap_eval(const int *leaves, DevTables<T> D, const int *beg, const int *end, const double *ctr,
                           const double *side, const int *lvl, const int *woff, const int *widx, const double *pos,
                           int64_t n, const cpx<T> *L, const cpx<T> *M, double *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int li = blockIdx.x;
    int b = leaves[li];
    const int p = D.p, nc = ncoef(p), P = p + 2, st = ncoef(P);
    T *smr = reinterpret_cast<T *>(smem_raw);
    Rec<T> R = load_rec(D, smr);   // recurrence tables cover degree p + 2
    Lad<T> G = load_lad(D, smr + rec_floats<T>(p));
    cpx<T> *EV = reinterpret_cast<cpx<T> *>(smr + tab_floats<T>(p));
    cpx<T> *tmp = EV + 13 * st;
    cpx<T> *srcs = tmp + 3 * st;
    double cbx = ctr[3 * b], cby = ctr[3 * b + 1], cbz = ctr[3 * b + 2];
    int j0 = beg[b], j1 = end[b];
    int nw = woff[li + 1] - woff[li];
    bool has_local = lvl[b] >= 2;
    for (int jc = j0; jc < j1; jc += blockDim.x) {
        int j = jc + threadIdx.x;
        bool act = j < j1;
        double x = act ? pos[j] : cbx, y = act ? pos[n + j] : cby, z = act ? pos[2 * n + j] : cbz;
        double res[kSets][13];
        for (int k = 0; k < kSets; ++k)
            for (int c = 0; c < 13; ++c) res[k][c] = 0;
        for (int w = -1; w < nw; ++w) {
            if (w < 0 && !has_local) continue;
            int C = w < 0 ? b : widx[woff[li] + w];
            const cpx<T> *E = w < 0 ? L + size_t(C) * kSets * nc : M + size_t(C) * kSets * nc;
            double h = side[C], ih = 1.0 / h;
            T vx = T((x - ctr[3 * C]) * ih), vy = T((y - ctr[3 * C + 1]) * ih), vz = T((z - ctr[3 * C + 2]) * ih);
            for (int k = 0; k < kSets; ++k) {
                __syncthreads();
                for (int i = threadIdx.x; i < nc; i += blockDim.x) srcs[i] = E[k * nc + i];
                __syncthreads();
                if (w < 0) build_lap_set<T, false>(srcs, p, P, EV, tmp, G);
                else build_lap_set<T, true>(srcs, p, P, EV, tmp, G);
                T acc[13];
#pragma unroll
                for (int q = 0; q < 13; ++q) acc[q] = 0;
                if (w < 0) eval_fields<T, 13, false>(vx, vy, vz, p, EV, st, R.a, R.b, R.c, acc);
                else eval_fields<T, 13, true>(vx, vy, vz, P, EV, st, R.a, R.b, R.c, acc);
                res[k][0] += ih * double(acc[0]);
                for (int c = 1; c < 4; ++c) res[k][c] += ih * ih * double(acc[c]);
                for (int c = 4; c < 13; ++c) res[k][c] += ih * ih * ih * double(acc[c]);
            }
        }
        if (act)
            for (int k = 0; k < kSets; ++k)
                for (int c = 0; c < 13; ++c) out[(size_t(j) * kSets + k) * 13 + c] = res[k][c];
    }
}

// ---------------------------------------------------------------- driver

template <typename T>
static size_t smem_p2x(int p, int threads) {
    const int nc = ncoef(p), chunk = p2x_chunk(p, threads);
    return sizeof(T) * ((rec_floats<T>(p) + 1) & ~1) + sizeof(cpx<T>) * (chunk * nc + 2 * kSets * nc) +
           sizeof(T) * 4 * chunk + 64;
}
template <typename T>
static size_t smem_m2x(int p, int s) {
    int nc = ncoef(p);
    return sizeof(cpx<T>) * (3 * kSets * nc + 2 * s * (kSets * (p + 1) + 1));
}
template <typename T>
static size_t smem_x2l(int p, int s, int NU) {
    int nc = ncoef(p);
    return sizeof(cpx<T>) * (4 * NU + 2 * s * (p + 1) + 4 * kSets * nc);
}
template <typename T>
static size_t smem_far(int p) {
    int st = ncoef(p + 2);
    return sizeof(T) * tab_floats<T>(p) + sizeof(cpx<T>) * (kNE * st + 4 * st + kSets * ncoef(p)) + 64;
}
template <typename T>
static size_t smem_lap(int p) {
    int st = ncoef(p + 2);
    return sizeof(T) * tab_floats<T>(p) + sizeof(cpx<T>) * (13 * st + 3 * st + ncoef(p)) + 64;
}

// Raise a kernel's dynamic shared-memory limit once per device and kernel
// (never while a stream is being captured: the first, uncaptured matvec sets
// every limit it needs).
static std::mutex g_smem_mu;
static std::map<std::pair<int, const void *>, size_t> g_smem_done;

template <typename K>
static int set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return RPY_OK;
    int dev = 0;
    RPY_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t &d = g_smem_done[{dev, reinterpret_cast<const void *>(kernel)}];
    if (bytes > d) {
        RPY_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
        d = bytes;
    }
    return RPY_OK;
}

// Threads of an X2X block: each handles elements e, e + blockDim, ... of the
// 4 S merged plane waves; the fewest warps that keep the number of rounds of
// 256 threads, so that the last round is not left nearly empty.
static int even_threads(int items) {
    const int rounds = (items + 255) / 256;
    return std::max(64, ((items + rounds - 1) / rounds + 31) / 32 * 32);
}
static int x2x_threads(int S) { return even_threads(kSets * S); }

template <typename T>
int run_far_t(Tree &t, const DevTables<T> &D, const double *fs, const double *lapq, double *ufar, double *lapout,
              const SysConst &sc, cudaStream_t st) {
    const int p = D.p, nc = ncoef(p);
    cpx<T> *M = static_cast<cpx<T> *>(t.M), *L = static_cast<cpx<T> *>(t.L);
    cpx<T> *Xo = static_cast<cpx<T> *>(t.Xo), *Xi = static_cast<cpx<T> *>(t.Xi);
    int nbx = t.nbox;
    RPY_CHECK(cudaMemsetAsync(L, 0, sizeof(cpx<T>) * size_t(nbx) * kSets * nc, st));
    if (t.nlevels <= 2) {
        // no box at level >= 2: nothing is far
        if (ufar) RPY_CHECK(cudaMemsetAsync(ufar, 0, sizeof(double) * 3 * size_t(t.n), st));
        if (lapout) RPY_CHECK(cudaMemsetAsync(lapout, 0, sizeof(double) * 52 * size_t(t.n), st));
        return RPY_OK;
    }
    int b2 = t.level_off[2];
    int n2 = nbx - b2;
    // origin of q4 (RPY charges only; the Laplace diagnostic takes its charges as given):
    // each expansion's own box centre by default in the FP32 form at 6 digits, the cube
    // centre otherwise (in FP64, and at 3 digits, its rounding stays far below the setting)
    const int fl = t.params.flags;
    const int rb = lapq ? 0
                        : (fl & RPY_FLAG_BOX_ORIGIN) ? 1
                        : (fl & RPY_FLAG_CUBE_ORIGIN) ? 0
                        : (sizeof(T) == 4 && t.params.digits >= 6);
    // upward pass
    size_t sp = smem_p2x<T>(p, 128);
    RPY_TRY(set_smem(k_p2x<T, 0>, sp));
    RPY_TRY(set_smem(k_p2x<T, 1>, sp));
    k_p2x<T, 0><<<n2, 128, sp, st>>>(b2, n2, D, t.b_begin, t.b_end, t.b_center, t.b_side, t.b_level, t.b_leaf,
                                     t.b_sys, t.x_off, t.x_idx, t.pos, fs, lapq, t.n, sc, M, rb);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_M2M, st);
    // FP64: rotation-based M2M and L2L (fewer FP64 operations).  FP32: the dense
    // operators below p = 12, the rotation forms (one child per block) from there
    const bool rot_l = sizeof(T) == 8 || p >= 12;
    size_t smr2 = sizeof(cpx<T>) * 3 * kSets * nc;
    int Dd = 2 * nc, thr = ((Dd + 31) / 32) * 32;
    size_t smd = sizeof(T) * kSets * Dd;
    RPY_TRY(set_smem(k_l2l_rot<T>, smr2));
    RPY_TRY(set_smem(k_m2m_child<T>, smr2));
    RPY_TRY(set_smem(k_m2m<T>, smd));
    RPY_TRY(set_smem(k_l2l<T>, smd));
    for (int l = t.nlevels - 2; l >= 2; --l) {
        int lb = t.level_off[l], ln = t.level_off[l + 1] - lb;
        if (ln > 0) {
            const int cb = t.level_off[l + 1], cn = t.level_off[l + 2] - cb;   // their children
            if (rot_l) {
                // the share slots exist whenever a level >= 2 does (tree_alloc_workspace)
                if (cn > 0) {
                    if (!t.m2m_scratch) return RPY_ERR_INTERNAL;
                    cpx<T> *Sc = static_cast<cpx<T> *>(t.m2m_scratch);
                    k_m2m_child<T><<<cn, 256, smr2, st>>>(cb, lb, D, t.b_parent, t.b_cell, t.b_side, rb, M, Sc);
                    k_m2m_sum<T><<<ln, 256, 0, st>>>(lb, kSets * nc, t.b_leaf, t.b_child, Sc, M);
                    RPY_LAUNCHED(2);
                }
            } else {
                k_m2m<T><<<ln, thr, smd, st>>>(lb, ln, D, t.b_leaf, t.b_child, t.b_side, rb, M);
                RPY_LAUNCHED(1);
            }
        }
    }
    RPY_CHECK(cudaGetLastError());
    // plane-wave M2L: all three frames in one pass, or (large trees, where the
    // plane-wave buffers of six directions would not fit) one frame per pass,
    // each pass adding its frame's share into L (with profiling on, every pass's
    // M2X, X2X and X2L launches are timed under their own stages).
    const int nf = t.x_frames;
    size_t smx = smem_m2x<T>(p, D.s);
    RPY_TRY(set_smem(k_m2x<T>, smx));
    size_t sxl = sizeof(T) == 4 ? smem_x2l4(p, D.s, D.S) : smem_x2l<T>(p, D.s, D.NU);
    if constexpr (sizeof(T) == 4) RPY_TRY(set_smem(k_x2l4, sxl));
    else RPY_TRY(set_smem(k_x2l<T>, sxl));
    for (int f0 = 0; f0 < 3; f0 += nf) {
        prof_mark(t, RPY_STAGE_M2X, st);
        k_m2x<T><<<n2, even_threads(sizeof(T) == 8 ? D.NU : D.S), smx, st>>>(b2, n2, D, M, Xo, f0, nf);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
        prof_mark(t, RPY_STAGE_X2X, st);
        if (t.n_x2x_par > 0) {
            dim3 g(t.n_x2x_par, 2 * nf);
            // FP32 (and the box-origin form): the four sets of a wave in one thread.  FP32 with
            // up to 256 stored waves: shifts from per-axis factors in shared memory (measured
            // faster there; at more waves the shared memory costs occupancy and the table is
            // faster)
            if (sizeof(T) == 4 && !rb && D.S <= 256) {
                // cube origin, few plane waves: one set per thread, shifts from per-axis factors
                const size_t sxx = sizeof(T) * ((6 * D.S + 3) & ~3) + 2 * sizeof(cpx<T>) * 6 * D.S;
                k_x2x<T, true><<<g, x2x_threads(D.S), sxx, st>>>(t.x2x_par, D, t.b_coll, t.b_child, t.b_leaf, Xo,
                                                                 Xi, f0, nf);
            } else if (sizeof(T) == 4 || rb) {
                bool fac = false;
                if constexpr (sizeof(T) == 4) {
                    if (D.S > 256 && D.S <= 480) {
                        // a producer warp stages the sources through shared memory by bulk copies
                        // (measured faster than per-thread loads from 323 stored waves up; at 3 digits,
                        // 134 waves, the per-thread loads below keep two to three blocks per SM and win)
                        const size_t sxx = x2x_tma_smem(D.S);
                        RPY_TRY(set_smem(k_x2x_tma, sxx));
                        k_x2x_tma<<<g, (D.S + 31) / 32 * 32 + 32, sxx, st>>>(t.x2x_par, D, t.b_coll, t.b_child,
                                                                             t.b_leaf, t.b_side, Xo, Xi, f0, nf, rb,
                                                                             t.dev_status);
                        fac = true;
                    } else if (D.S <= 256) {
                        const size_t sxx = sizeof(T) * ((6 * D.S + 3) & ~3) + 2 * sizeof(cpx<T>) * 6 * D.S;
                        k_x2x4<T, true><<<g, even_threads(D.S), sxx, st>>>(t.x2x_par, D, t.b_coll, t.b_child,
                                                                           t.b_leaf, t.b_side, Xo, Xi, f0, nf, rb);
                        fac = true;
                    }
                }
                if (!fac) {
                    k_x2x4<T, false><<<g, even_threads(D.S), 0, st>>>(t.x2x_par, D, t.b_coll, t.b_child, t.b_leaf,
                                                                      t.b_side, Xo, Xi, f0, nf, rb);
                }
            } else {
                k_x2x<T, false><<<g, x2x_threads(D.S), 0, st>>>(t.x2x_par, D, t.b_coll, t.b_child, t.b_leaf, Xo, Xi,
                                                                f0, nf);
            }
            RPY_LAUNCHED(1);
            RPY_CHECK(cudaGetLastError());
        }
        prof_mark(t, RPY_STAGE_X2L, st);
        // FP32 X2L: blocks sized to the (node, m) items of its widest phase at low
        // order; at high order the shared memory already limits the blocks per SM
        // and 256 threads hide latency better
        const int tx = D.s * (p + 1) <= 256 ? even_threads(D.s * (p + 1)) : 256;
        if constexpr (sizeof(T) == 4) k_x2l4<<<n2, tx, sxl, st>>>(b2, n2, D, Xi, L, f0, nf);
        else k_x2l<T><<<n2, 256, sxl, st>>>(b2, n2, D, Xi, L, f0, nf);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
    }
    // X list
    prof_mark(t, RPY_STAGE_P2L, st);
    k_p2x<T, 1><<<n2, 128, sp, st>>>(b2, n2, D, t.b_begin, t.b_end, t.b_center, t.b_side, t.b_level, t.b_leaf,
                                     t.b_sys, t.x_off, t.x_idx, t.pos, fs, lapq, t.n, sc, L, rb);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    // downward pass
    prof_mark(t, RPY_STAGE_L2L, st);
    for (int l = 3; l < t.nlevels; ++l) {
        int lb = t.level_off[l], ln = t.level_off[l + 1] - lb;
        if (ln > 0) {
            if (rot_l) k_l2l_rot<T><<<ln, 256, smr2, st>>>(lb, ln, D, t.b_parent, t.b_cell, t.b_side, rb, L);
            else k_l2l<T><<<ln, thr, smd, st>>>(lb, ln, D, t.b_parent, t.b_cell, t.b_side, rb, L);
            RPY_LAUNCHED(1);
        }
    }
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_EVAL, st);
    if (ufar) {
        cpx<T> *EVg = static_cast<cpx<T> *>(t.EVg);
        size_t sp2 = sizeof(T) * (((6 * ncoef(p + 2) + 1) & ~1)) + sizeof(cpx<T>) * 2 * kSets * nc + 64;
        RPY_TRY(set_smem(k_eval_prep<T>, sp2));
        // one expansion per velocity component unless the per-potential form is asked for
        const int per_comp = (t.params.flags & RPY_FLAG_EVAL_PER_POTENTIAL) ? 0 : 1;
        k_eval_prep<T><<<t.nleaf, 128, sp2, st>>>(t.leaves, D, t.b_center, t.b_level, t.b_sys, sc, L, EVg, per_comp,
                                                  rb);
        RPY_LAUNCHED(1);
        const int ga = int((t.n + 127) / 128);
        if (per_comp)
            k_eval_apply<T, kNF2><<<ga, 128, 0, st>>>(t.n, t.bead_leaf, t.leaves, D, t.b_center, t.b_side, t.b_level,
                                                      t.b_sys, t.pos, sc, EVg, ufar);
        else
            k_eval_apply<T, kNF><<<ga, 128, 0, st>>>(t.n, t.bead_leaf, t.leaves, D, t.b_center, t.b_side, t.b_level,
                                                     t.b_sys, t.pos, sc, EVg, ufar);
        RPY_LAUNCHED(1);
        size_t sf = smem_far<T>(p);
        RPY_TRY(set_smem(k_far_eval<T>, sf));
        k_far_eval<T><<<t.nleaf, 64, sf, st>>>(t.leaves, D, t.b_begin, t.b_end, t.b_center, t.b_side, t.b_level,
                                                t.b_sys, t.w_off, t.w_idx, t.pos, t.n, sc, L, M, ufar, rb);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
    }
    if (lapout) {
        size_t sl = smem_lap<T>(p);
        RPY_TRY(set_smem(k_lap_eval<T>, sl));
        k_lap_eval<T><<<t.nleaf, 64, sl, st>>>(t.leaves, D, t.b_begin, t.b_end, t.b_center, t.b_side, t.b_level,
                                                t.w_off, t.w_idx, t.pos, t.n, L, M, lapout);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
    }
    return RPY_OK;
}

template int run_far_t<double>(Tree &, const DevTables<double> &, const double *, const double *, double *, double *,
                               const SysConst &, cudaStream_t);
template int run_far_t<float>(Tree &, const DevTables<float> &, const double *, const double *, double *, double *,
                              const SysConst &, cudaStream_t);

}  // namespace rpy
