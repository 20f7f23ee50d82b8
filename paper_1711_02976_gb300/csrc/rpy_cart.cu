// Polynomial (Cartesian Taylor) far field: the alternative to spherical-harmonic
// and plane-wave expansions that the paper's conclusion (Sec. 5) proposes for the
// low-accuracy setting, where polynomials evaluate faster than harmonics and
// exponentials.  Selected per tree by RPY_FLAG_CARTESIAN.
//
// Expansions of total degree <= P in the box-scaled offset eta = (r - c) / h of
// each box (c its centre, h its side), four charge sets (Sec. 2: q_1..3 = F,
// q_4 = F . (r - c), the fourth about the expansion's own centre):
//   multipole  M_b   = sum_j q_j eta_j^b                        (b a multi-index)
//   local      phi(x) = sum_a L_a eta^a,   eta = (x - c_T) / h
// Operators:
//   P2M   the sums above over a leaf's beads;
//   M2M   eta_P = eta_C / 2 + d, d = (c_C - c_P) / h_P = +-1/4 per axis:
//         M_a(P) += sum_{b <= a} prod_i C(a_i, b_i) 2^-b_i d_i^(a_i - b_i) M_b(C);
//   M2L   for a V-list source S of T at the same level, R = (c_T - c_S) / h (an
//         integer vector in [-3, 3]^3), with t_g(R) the Taylor coefficients of
//         1/|R + y| in y:
//         L_a(T) += (1/h) sum_{|a + b| <= P} (-1)^|b| prod_i C(a_i + b_i, b_i) t_{a+b}(R) M_b(S);
//   L2L   eta_P = eta_C / 2 + d:
//         L_a(C) += 2^-|a| sum_{b >= a} prod_i C(b_i, a_i) d_i^(b_i - a_i) L_b(P);
//   the fourth set moves its origin with every translation, M4(o') = M4(o) + (o - o') . M_F;
//   L2P   Eq. (2.8) at coefficient level: with P_kd[b] = (b_d + 1) L_k[b + e_d] (the
//         eta-derivative of L_k) and Q = sum_k P_kk,
//         U_d[a] = C1 L_d[a] - C1 sum_k P_kd[a - e_k] + (C1/h) P_4d[a] - (C2/h^2) (a_d + 1) Q[a + e_d],
//         u_d(x) = sum_a U_d[a] eta^a: three polynomials per leaf, evaluated per bead.
// Multipoles are stored [box][monomial][4 sets] (one 16-byte load per monomial in FP32),
// locals [box][4 sets][monomial].  The M2L terms of each a form a prefix of the graded
// monomials b (those with |b| <= P - |a|), and each V-list offset's operator values
// c_ab t_{a+b}(R) are tabulated per offset, so a term costs one table load, one multipole
// load and four FMAs.
// W- and X-list interactions are all summed directly (the tree's direct
// substitutes), so M2P and P2L are not needed.  The Taylor coefficients of 1/|R + y|
// follow the recurrence |g| |R|^2 t_g = -(2|g| - 1) sum_i R_i t_{g - e_i} - (|g| - 1) sum_i t_{g - 2 e_i}.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rpy_internal.h"

namespace rpy {

// ---------------------------------------------------------------- host tables
namespace {

constexpr int kCartRun = 16;    // M2L pairs per work item
constexpr int kCartItems = 4;   // work items per M2L thread (items <= kCartItems x threads)

struct CartHost {
    int P = 0, N = 0;
    std::vector<int> ex;                  // [N][3] exponents, graded order
    std::vector<int> idx3;                // [(P+1)^3] monomial index of (a, b, c), -1 beyond degree P
    std::vector<int> m2l_off, m2l_b, m2l_g;   // pairs (a, b), |a + b| <= P, grouped by a
    std::vector<double> m2l_c;            // (-1)^|b| prod C(a_i + b_i, b_i)
    // M2L work items: the pairs of each a in runs of at most kCartRun (balanced threads);
    // item i covers pairs [it_k0[i], it_k0[i + 1]) of monomial it_a[i]; items of a are
    // [it_of[a], it_of[a + 1])
    std::vector<int> it_a, it_k0, it_of;
    std::vector<double> dtab;             // [343][N] t_g(R), R = (i - 3, j - 3, k - 3), index 49 i + 7 j + k
    std::vector<double> ktab;             // [343][pairs] c_ab t_{a+b}(R): the M2L operator per offset
    std::vector<int> mm_off, mm_b, mm_odd;    // M2M pairs (a, b <= a), odd-exponent mask of a - b
    std::vector<double> mm_c;             // prod C(a_i, b_i) 2^-b_i 4^-(a_i - b_i)
    std::vector<int> ll_off, ll_b, ll_odd;    // L2L pairs (a, b >= a)
    std::vector<double> ll_c;             // 2^-|a| prod C(b_i, a_i) 4^-(b_i - a_i)
};

double binom(int n, int k) {
    double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

void build_cart(int P, CartHost &h) {
    h.P = P;
    const int P1 = P + 1;
    h.idx3.assign(P1 * P1 * P1, -1);
    for (int n = 0; n <= P; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                const int c = n - a - b;
                h.idx3[(a * P1 + b) * P1 + c] = int(h.ex.size() / 3);
                h.ex.insert(h.ex.end(), {a, b, c});
            }
    h.N = int(h.ex.size() / 3);
    const int N = h.N;
    auto id = [&](int a, int b, int c) { return (a < 0 || b < 0 || c < 0 || a + b + c > P) ? -1 : h.idx3[(a * P1 + b) * P1 + c]; };
    // M2L pairs
    h.m2l_off.push_back(0);
    for (int i = 0; i < N; ++i) {
        const int *A = &h.ex[3 * i];
        for (int j = 0; j < N; ++j) {
            const int *B = &h.ex[3 * j];
            const int g = id(A[0] + B[0], A[1] + B[1], A[2] + B[2]);
            if (g < 0) continue;
            double c = ((B[0] + B[1] + B[2]) & 1) ? -1.0 : 1.0;
            for (int d = 0; d < 3; ++d) c *= binom(A[d] + B[d], B[d]);
            h.m2l_b.push_back(j);
            h.m2l_g.push_back(g);
            h.m2l_c.push_back(c);
        }
        h.m2l_off.push_back(int(h.m2l_b.size()));
    }
    for (int i = 0; i < N; ++i) {
        h.it_of.push_back(int(h.it_a.size()));
        for (int k = h.m2l_off[i]; k < h.m2l_off[i + 1]; k += kCartRun) {
            h.it_a.push_back(i);
            h.it_k0.push_back(k);
        }
    }
    h.it_of.push_back(int(h.it_a.size()));
    h.it_k0.push_back(h.m2l_off[N]);
    // Taylor coefficients of 1/|R + y| for the 343 integer offsets
    h.dtab.assign(size_t(343) * N, 0.0);
    for (int oi = 0; oi < 343; ++oi) {
        const double R[3] = {double(oi / 49 - 3), double((oi / 7) % 7 - 3), double(oi % 7 - 3)};
        const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
        if (r2 == 0) continue;
        double *t = &h.dtab[size_t(oi) * N];
        t[0] = 1.0 / std::sqrt(r2);
        for (int g = 1; g < N; ++g) {
            const int *G = &h.ex[3 * g];
            const int n = G[0] + G[1] + G[2];
            double s = 0;
            for (int d = 0; d < 3; ++d) {
                int E1[3] = {G[0], G[1], G[2]};
                if (E1[d] >= 1) {
                    E1[d] -= 1;
                    s -= (2 * n - 1) * R[d] * t[id(E1[0], E1[1], E1[2])];
                }
                int E2[3] = {G[0], G[1], G[2]};
                if (E2[d] >= 2) {
                    E2[d] -= 2;
                    s -= (n - 1) * t[id(E2[0], E2[1], E2[2])];
                }
            }
            t[g] = s / (n * r2);
        }
    }
    const size_t npair = h.m2l_b.size();
    h.ktab.assign(size_t(343) * npair, 0.0);
    for (int oi = 0; oi < 343; ++oi)
        for (size_t k = 0; k < npair; ++k)
            h.ktab[oi * npair + k] = h.m2l_c[k] * h.dtab[size_t(oi) * N + h.m2l_g[k]];
    // M2M and L2L pairs (octant signs applied on the device through the odd masks)
    h.mm_off.push_back(0);
    h.ll_off.push_back(0);
    for (int i = 0; i < N; ++i) {
        const int *A = &h.ex[3 * i];
        for (int j = 0; j < N; ++j) {
            const int *B = &h.ex[3 * j];
            if (B[0] <= A[0] && B[1] <= A[1] && B[2] <= A[2]) {
                double c = 1;
                int odd = 0;
                for (int d = 0; d < 3; ++d) {
                    c *= binom(A[d], B[d]) * std::ldexp(1.0, -B[d]) * std::ldexp(1.0, -2 * (A[d] - B[d]));
                    if ((A[d] - B[d]) & 1) odd |= 1 << d;
                }
                h.mm_b.push_back(j);
                h.mm_c.push_back(c);
                h.mm_odd.push_back(odd);
            }
            if (B[0] >= A[0] && B[1] >= A[1] && B[2] >= A[2]) {
                double c = std::ldexp(1.0, -(A[0] + A[1] + A[2]));
                int odd = 0;
                for (int d = 0; d < 3; ++d) {
                    c *= binom(B[d], A[d]) * std::ldexp(1.0, -2 * (B[d] - A[d]));
                    if ((B[d] - A[d]) & 1) odd |= 1 << d;
                }
                h.ll_b.push_back(j);
                h.ll_c.push_back(c);
                h.ll_odd.push_back(odd);
            }
        }
        h.mm_off.push_back(int(h.mm_b.size()));
        h.ll_off.push_back(int(h.ll_b.size()));
    }
}

template <typename T>
struct CartDev {
    int P, N;
    const int *ex, *idx3;
    const int *m2l_off, *m2l_b, *m2l_g;
    const T *m2l_c, *dtab;
    const int *it_a, *it_k0, *it_of;
    int n_items, n_pairs;
    const T *ktab;
    const int *mm_off, *mm_b, *mm_odd;
    const T *mm_c;
    const int *ll_off, *ll_b, *ll_odd;
    const T *ll_c;
};

struct CartDevSet {
    void *mem = nullptr;
    CartDev<double> d64{};
    CartDev<float> d32{};
};

std::mutex g_cart_mu;
std::map<std::pair<int, int>, CartDevSet *> g_cart;   // (device, P), kept for the process

template <typename T>
void pack(const CartHost &h, std::vector<char> &blob, std::vector<size_t> &o) {
    auto put = [&](const void *src, size_t bytes) {
        size_t off = (blob.size() + 255) / 256 * 256;
        blob.resize(off + bytes);
        if (bytes) std::memcpy(blob.data() + off, src, bytes);
        o.push_back(off);
    };
    auto putI = [&](const std::vector<int> &v) { put(v.data(), sizeof(int) * v.size()); };
    auto putT = [&](const std::vector<double> &v) {
        std::vector<T> c(v.begin(), v.end());
        put(c.data(), sizeof(T) * c.size());
    };
    putI(h.ex);        // 0
    putI(h.idx3);      // 1
    putI(h.m2l_off);   // 2
    putI(h.m2l_b);     // 3
    putI(h.m2l_g);     // 4
    putT(h.m2l_c);     // 5
    putT(h.dtab);      // 6
    putI(h.mm_off);    // 7
    putI(h.mm_b);      // 8
    putI(h.mm_odd);    // 9
    putT(h.mm_c);      // 10
    putI(h.ll_off);    // 11
    putI(h.ll_b);      // 12
    putI(h.ll_odd);    // 13
    putT(h.ll_c);      // 14
    putI(h.it_a);      // 15
    putI(h.it_k0);     // 16
    putI(h.it_of);     // 17
    putT(h.ktab);      // 18
}

template <typename T>
CartDev<T> bind(const CartHost &h, const char *base, const std::vector<size_t> &o) {
    CartDev<T> d{};
    d.P = h.P;
    d.N = h.N;
    d.ex = reinterpret_cast<const int *>(base + o[0]);
    d.idx3 = reinterpret_cast<const int *>(base + o[1]);
    d.m2l_off = reinterpret_cast<const int *>(base + o[2]);
    d.m2l_b = reinterpret_cast<const int *>(base + o[3]);
    d.m2l_g = reinterpret_cast<const int *>(base + o[4]);
    d.m2l_c = reinterpret_cast<const T *>(base + o[5]);
    d.dtab = reinterpret_cast<const T *>(base + o[6]);
    d.mm_off = reinterpret_cast<const int *>(base + o[7]);
    d.mm_b = reinterpret_cast<const int *>(base + o[8]);
    d.mm_odd = reinterpret_cast<const int *>(base + o[9]);
    d.mm_c = reinterpret_cast<const T *>(base + o[10]);
    d.ll_off = reinterpret_cast<const int *>(base + o[11]);
    d.ll_b = reinterpret_cast<const int *>(base + o[12]);
    d.ll_odd = reinterpret_cast<const int *>(base + o[13]);
    d.ll_c = reinterpret_cast<const T *>(base + o[14]);
    d.it_a = reinterpret_cast<const int *>(base + o[15]);
    d.it_k0 = reinterpret_cast<const int *>(base + o[16]);
    d.it_of = reinterpret_cast<const int *>(base + o[17]);
    d.n_items = int(h.it_a.size());
    d.n_pairs = int(h.m2l_b.size());
    d.ktab = reinterpret_cast<const T *>(base + o[18]);
    return d;
}

int cart_tables(int dev, int P, CartDevSet **out) {
    std::lock_guard<std::mutex> lk(g_cart_mu);
    auto it = g_cart.find({dev, P});
    if (it != g_cart.end()) {
        *out = it->second;
        return RPY_OK;
    }
    CartHost h;
    build_cart(P, h);
    std::vector<char> b64, b32;
    std::vector<size_t> o64, o32;
    pack<double>(h, b64, o64);
    pack<float>(h, b32, o32);
    const size_t off32 = (b64.size() + 255) / 256 * 256;
    void *mem = nullptr;
    RPY_CHECK(cudaMalloc(&mem, off32 + b32.size()));
    cudaError_t e1 = cudaMemcpy(mem, b64.data(), b64.size(), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(static_cast<char *>(mem) + off32, b32.data(), b32.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFree(mem);
        return check_cuda("Cartesian table upload", e1 != cudaSuccess ? e1 : e2);
    }
    auto *s = new CartDevSet();
    s->mem = mem;
    s->d64 = bind<double>(h, static_cast<char *>(mem), o64);
    s->d32 = bind<float>(h, static_cast<char *>(mem) + off32, o32);
    g_cart[{dev, P}] = s;
    *out = s;
    return RPY_OK;
}

}  // namespace

int cart_terms(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// ---------------------------------------------------------------- kernels
namespace {

constexpr int kCartChunk = 64;   // beads staged per P2M round

// the four sets of one monomial from a 16-byte aligned [monomial][4 sets] array
__device__ __forceinline__ void load4(const float *p, float (&m)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    m[0] = v.x;
    m[1] = v.y;
    m[2] = v.z;
    m[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double (&m)[4]) {
    const double2 v = reinterpret_cast<const double2 *>(p)[0], w = reinterpret_cast<const double2 *>(p)[1];
    m[0] = v.x;
    m[1] = v.y;
    m[2] = w.x;
    m[3] = w.y;
}

// P2M: one block per leaf at level >= 2; thread = monomial a (four sets); beads
// staged with their powers of eta per axis; chunk sums enter the running sums by
// compensated addition in FP32.
template <typename T>
__global__ void k_cart_p2m(int b0, int nb, CartDev<T> D, const int *beg, const int *end, const double *ctr,
                           const double *side, const int *lvl, const int *leaf, const double *pos, const double *fs,
                           int64_t n, T *M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = b0 + blockIdx.x;
    if (lvl[b] < 2 || !leaf[b]) return;
    const int P = D.P, N = D.N, P1 = P + 1;
    T *pw = reinterpret_cast<T *>(smem_raw);          // [chunk][3][P1]
    T *qs = pw + kCartChunk * 3 * P1;                 // [chunk][4]
    const double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2], ih = 1.0 / side[b];
    const int a = threadIdx.x;
    int ea = 0, eb = 0, ec = 0;
    if (a < N) {
        ea = D.ex[3 * a];
        eb = D.ex[3 * a + 1];
        ec = D.ex[3 * a + 2];
    }
    T acc[kSets] = {0, 0, 0, 0}, cmp[kSets] = {0, 0, 0, 0};
    for (int j0 = beg[b]; j0 < end[b]; j0 += kCartChunk) {
        const int cnt = min(kCartChunk, end[b] - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int j = j0 + t;
            const double x = pos[j] - cx, y = pos[n + j] - cy, z = pos[2 * n + j] - cz;
            const double fx = fs[j], fy = fs[n + j], fz = fs[2 * n + j];
            const T e[3] = {T(x * ih), T(y * ih), T(z * ih)};
            for (int d = 0; d < 3; ++d) {
                T v = 1;
                for (int k = 0; k <= P; ++k) {
                    pw[(t * 3 + d) * P1 + k] = v;
                    v *= e[d];
                }
            }
            qs[4 * t] = T(fx);
            qs[4 * t + 1] = T(fy);
            qs[4 * t + 2] = T(fz);
            qs[4 * t + 3] = T(fx * x + fy * y + fz * z);   // q4 about the leaf's centre
        }
        __syncthreads();
        if (a < N) {
            T s[kSets] = {0, 0, 0, 0};
            for (int t = 0; t < cnt; ++t) {
                const T m = pw[(t * 3) * P1 + ea] * pw[(t * 3 + 1) * P1 + eb] * pw[(t * 3 + 2) * P1 + ec];
#pragma unroll
                for (int k = 0; k < kSets; ++k) s[k] = fma(qs[4 * t + k], m, s[k]);
            }
#pragma unroll
            for (int k = 0; k < kSets; ++k) {
                if constexpr (sizeof(T) == 4) {
                    const T yv = s[k] - cmp[k], tv = acc[k] + yv;
                    cmp[k] = (tv - acc[k]) - yv;
                    acc[k] = tv;
                } else {
                    acc[k] += s[k];
                }
            }
        }
    }
    if (a < N)
        for (int k = 0; k < kSets; ++k) M[(size_t(b) * N + a) * kSets + k] = acc[k];
}

// M2M: one block per parent (levels >= 2 with children); thread = monomial a.
template <typename T>
__global__ void k_cart_m2m(int b0, int nb, CartDev<T> D, const int *leaf, const int *child, const int *cell,
                           const double *side, T *M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = b0 + blockIdx.x;
    if (leaf[b]) return;
    const int N = D.N;
    T *Mc = reinterpret_cast<T *>(smem_raw);   // [4][N]
    const int a = threadIdx.x;
    const double hq = 0.25 * side[b];           // |c_C - c_P| per axis
    T acc[kSets] = {0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
        const int c = child[8 * b + o];
        if (c < 0) continue;   // block-uniform
        __syncthreads();
        for (int i = threadIdx.x; i < kSets * N; i += blockDim.x) Mc[i] = M[size_t(c) * kSets * N + i];
        __syncthreads();
        if (a < N) {
            T s[kSets] = {0, 0, 0, 0};
            const int neg = ~o & 7;   // axes where c_C - c_P < 0
            for (int k = D.mm_off[a]; k < D.mm_off[a + 1]; ++k) {
                const int bi = D.mm_b[k];
                const T cf = (__popc(D.mm_odd[k] & neg) & 1) ? -D.mm_c[k] : D.mm_c[k];
#pragma unroll
                for (int q = 0; q < kSets; ++q) s[q] = fma(cf, Mc[bi * kSets + q], s[q]);
            }
            // the fourth set about the parent's centre: + (c_C - c_P) . M_F
            const T dx = T((o & 1) ? hq : -hq), dy = T((o & 2) ? hq : -hq), dz = T((o & 4) ? hq : -hq);
            acc[0] += s[0];
            acc[1] += s[1];
            acc[2] += s[2];
            acc[3] += fma(dz, s[2], fma(dy, s[1], fma(dx, s[0], s[3])));
        }
    }
    if (a < N)
        for (int q = 0; q < kSets; ++q) M[(size_t(b) * N + a) * kSets + q] = acc[q];
}

// M2L over the V list: one block per target box at level >= 2.  The terms of each
// monomial a (b = 0 .. N_{P-|a|} - 1 in graded order) are split into work items of at
// most kCartRun terms; each thread keeps the partial sums of its items (up to
// kCartItems) over all sources in registers, and the items of each a are added in a
// fixed order at the end (deterministic).  Each source's multipole ([monomial][4 sets],
// set 4 moved to the target's centre) is staged in shared memory; the operator values
// c_ab t_{a+b}(R) of its offset come from the per-offset table.
template <typename T>
__global__ void k_cart_m2l(int b0, int nb, CartDev<T> D, const int *voff, const int *vidx, const int *cell,
                           const double *side, const int *lvl, T *M, T *L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = b0 + blockIdx.x;
    if (lvl[b] < 2) return;
    const int nv = voff[b + 1] - voff[b];
    if (nv == 0) return;
    const int N = D.N, NI = D.n_items, NP = D.n_pairs;
    T *Ms = reinterpret_cast<T *>(smem_raw);   // [N][4]
    T *part = Ms + kSets * N;                   // [NI][4]
    const double h = side[b];
    // this thread's items: first term, term count, first b
    int k0[kCartItems], kn[kCartItems], bb[kCartItems];
#pragma unroll
    for (int r = 0; r < kCartItems; ++r) {
        const int it = threadIdx.x + r * blockDim.x;
        k0[r] = 0;
        kn[r] = 0;
        bb[r] = 0;
        if (it < NI) {
            k0[r] = D.it_k0[it];
            kn[r] = D.it_k0[it + 1] - k0[r];
            bb[r] = k0[r] - D.m2l_off[D.it_a[it]];
        }
    }
    T acc[kCartItems][kSets];
#pragma unroll
    for (int r = 0; r < kCartItems; ++r)
#pragma unroll
        for (int q = 0; q < kSets; ++q) acc[r][q] = 0;
    for (int v = 0; v < nv; ++v) {
        const int S = vidx[voff[b] + v];
        // R = (c_T - c_S) / h from the integer cells (same level)
        const int rx = cell[3 * b] - cell[3 * S], ry = cell[3 * b + 1] - cell[3 * S + 1],
                  rz = cell[3 * b + 2] - cell[3 * S + 2];
        const T *kt = D.ktab + size_t((rx + 3) * 49 + (ry + 3) * 7 + (rz + 3)) * NP;
        // the fourth set about the target's centre: + (c_S - c_T) . M_F = -h R . M_F
        const T dx = T(-h * rx), dy = T(-h * ry), dz = T(-h * rz);
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const T *src = M + (size_t(S) * N + i) * kSets;
            const T m0 = src[0], m1 = src[1], m2 = src[2];
            Ms[kSets * i] = m0;
            Ms[kSets * i + 1] = m1;
            Ms[kSets * i + 2] = m2;
            Ms[kSets * i + 3] = fma(dz, m2, fma(dy, m1, fma(dx, m0, src[3])));
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kCartItems; ++r) {
            for (int i = 0; i < kn[r]; ++i) {
                const T cf = kt[k0[r] + i];
                T m[kSets];
                load4(Ms + kSets * (bb[r] + i), m);
#pragma unroll
                for (int q = 0; q < kSets; ++q) acc[r][q] = fma(cf, m[q], acc[r][q]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kCartItems; ++r) {
        const int it = threadIdx.x + r * blockDim.x;
        if (it < NI)
            for (int q = 0; q < kSets; ++q) part[it * kSets + q] = acc[r][q];
    }
    __syncthreads();
    const T ih = T(1.0 / h);
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
        T s[kSets] = {0, 0, 0, 0};
        for (int it = D.it_of[a]; it < D.it_of[a + 1]; ++it)
            for (int q = 0; q < kSets; ++q) s[q] += part[it * kSets + q];
        for (int q = 0; q < kSets; ++q) L[(size_t(b) * kSets + q) * N + a] += ih * s[q];
    }
}

// L2L: one block per child box (level >= 3); thread = monomial a.
template <typename T>
__global__ void k_cart_l2l(int b0, int nb, CartDev<T> D, const int *par, const int *cell, const double *side, T *L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = b0 + blockIdx.x;
    const int Pb = par[b];
    const int N = D.N;
    T *Lp = reinterpret_cast<T *>(smem_raw);   // [4][N]
    for (int i = threadIdx.x; i < kSets * N; i += blockDim.x) Lp[i] = L[size_t(Pb) * kSets * N + i];
    __syncthreads();
    const int a = threadIdx.x;
    if (a >= N) return;
    const int o = (cell[3 * b] & 1) | ((cell[3 * b + 1] & 1) << 1) | ((cell[3 * b + 2] & 1) << 2);
    const int neg = ~o & 7;
    T s[kSets] = {0, 0, 0, 0};
    for (int k = D.ll_off[a]; k < D.ll_off[a + 1]; ++k) {
        const int bi = D.ll_b[k];
        const T cf = (__popc(D.ll_odd[k] & neg) & 1) ? -D.ll_c[k] : D.ll_c[k];
#pragma unroll
        for (int q = 0; q < kSets; ++q) s[q] = fma(cf, Lp[q * N + bi], s[q]);
    }
    // the fourth set about the child's centre: + (c_P - c_C) . L_F
    const double hh = 0.5 * side[b];
    const T dx = T((o & 1) ? -hh : hh), dy = T((o & 2) ? -hh : hh), dz = T((o & 4) ? -hh : hh);
    T *dst = L + size_t(b) * kSets * N;
    dst[a] += s[0];
    dst[N + a] += s[1];
    dst[2 * N + a] += s[2];
    dst[3 * N + a] += fma(dz, s[2], fma(dy, s[1], fma(dx, s[0], s[3])));
}

// Eq. (2.8) at coefficient level: three velocity polynomials per leaf at level >= 2.
template <typename T>
__global__ void k_cart_prep(const int *leaves, CartDev<T> D, const double *side, const int *lvl, const int *bsys,
                            SysConst sc, const T *L, T *U) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int li = blockIdx.x, b = leaves[li];
    if (lvl[b] < 2) return;
    const int P = D.P, N = D.N, P1 = P + 1;
    T *Ls = reinterpret_cast<T *>(smem_raw);
    for (int i = threadIdx.x; i < kSets * N; i += blockDim.x) Ls[i] = L[size_t(b) * kSets * N + i];
    __syncthreads();
    const int sy = bsys[b];
    const double h = side[b];
    const T c1 = T(sc.pc[sy].C1), c1h = T(sc.pc[sy].C1 / h), c2h = T(sc.pc[sy].C2 / (h * h));
    auto at = [&](int q, int e0, int e1, int e2) -> T {   // L_q[e], 0 beyond degree P
        if (e0 + e1 + e2 > P) return T(0);
        return Ls[q * N + D.idx3[(e0 * P1 + e1) * P1 + e2]];
    };
    // derivative of L_q along axis d at exponent e: (e_d + 1) L_q[e + e_d]
    auto der = [&](int q, int d, int e0, int e1, int e2) -> T {
        if (e0 < 0 || e1 < 0 || e2 < 0) return T(0);
        const int E[3] = {e0 + (d == 0), e1 + (d == 1), e2 + (d == 2)};
        return T(E[d]) * at(q, E[0], E[1], E[2]);
    };
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
        const int e0 = D.ex[3 * a], e1 = D.ex[3 * a + 1], e2 = D.ex[3 * a + 2];
        for (int d = 0; d < 3; ++d) {
            T u = c1 * at(d, e0, e1, e2);
            // - C1 sum_k eta_k P_kd: coefficient at a takes P_kd[a - e_k]
            T xs = der(0, d, e0 - 1, e1, e2) + der(1, d, e0, e1 - 1, e2) + der(2, d, e0, e1, e2 - 1);
            u = fma(-c1, xs, u);
            u = fma(c1h, der(3, d, e0, e1, e2), u);
            // Q[a + e_d] (a_d + 1): Q[e] = sum_k (e_k + 1) L_k[e + e_k]
            const int E[3] = {e0 + (d == 0), e1 + (d == 1), e2 + (d == 2)};
            T Qv = 0;
            if (E[0] + E[1] + E[2] <= P)
                Qv = der(0, 0, E[0], E[1], E[2]) + der(1, 1, E[0], E[1], E[2]) + der(2, 2, E[0], E[1], E[2]);
            u = fma(-c2h, T(E[d]) * Qv, u);
            U[(size_t(li) * 3 + d) * N + a] = u;
        }
    }
}

// One thread per bead: the leaf's three velocity polynomials at eta, the
// monomials formed by running products in (a, b, c) order.
template <typename T>
__global__ void k_cart_apply(int64_t n, const int *bead_leaf, const int *leaves, CartDev<T> D, const double *ctr,
                             const double *side, const int *lvl, const double *pos, const T *U, double *ufar) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int li = bead_leaf[i], b = leaves[li];
    double u[3] = {0, 0, 0};
    if (lvl[b] >= 2) {
        const int P = D.P, N = D.N, P1 = P + 1;
        const double ih = 1.0 / side[b];
        const T ex = T((pos[i] - ctr[3 * b]) * ih), ey = T((pos[n + i] - ctr[3 * b + 1]) * ih),
                ez = T((pos[2 * n + i] - ctr[3 * b + 2]) * ih);
        const T *Ub = U + size_t(li) * 3 * N;
        T s0 = 0, s1 = 0, s2 = 0;
        T xa = 1;
        for (int a = 0; a <= P; ++a) {
            T xy = xa;
            for (int bb = 0; bb <= P - a; ++bb) {
                T m = xy;
                const int *row = D.idx3 + (a * P1 + bb) * P1;
                for (int c = 0; c <= P - a - bb; ++c) {
                    const int k = row[c];
                    s0 = fma(Ub[k], m, s0);
                    s1 = fma(Ub[N + k], m, s1);
                    s2 = fma(Ub[2 * N + k], m, s2);
                    m *= ez;
                }
                xy *= ey;
            }
            xa *= ex;
        }
        u[0] = double(s0);
        u[1] = double(s1);
        u[2] = double(s2);
    }
    for (int d = 0; d < 3; ++d) ufar[3 * i + d] = u[d];
}

}  // namespace

// ---------------------------------------------------------------- driver
// Raise a kernel's dynamic shared-memory limit when it needs more than 48 KB.
template <typename K>
static int set_cart_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return RPY_OK;
    RPY_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    return RPY_OK;
}

template <typename T>
int run_cart_t(Tree &t, const double *fs, double *ufar, const SysConst &sc, cudaStream_t st) {
    CartDevSet *set = nullptr;
    RPY_TRY(cart_tables(t.device, t.p, &set));
    const CartDev<T> D = sizeof(T) == 8 ? *reinterpret_cast<const CartDev<T> *>(&set->d64)
                                        : *reinterpret_cast<const CartDev<T> *>(&set->d32);
    const int N = D.N, nbx = t.nbox;
    T *M = static_cast<T *>(t.M), *L = static_cast<T *>(t.L), *U = static_cast<T *>(t.EVg);
    RPY_CHECK(cudaMemsetAsync(L, 0, sizeof(T) * size_t(nbx) * kSets * N, st));
    if (t.nlevels <= 2) {
        RPY_CHECK(cudaMemsetAsync(ufar, 0, sizeof(double) * 3 * size_t(t.n), st));
        return RPY_OK;
    }
    const int b2 = t.level_off[2], n2 = nbx - b2;
    const int thr = (N + 31) / 32 * 32;
    const size_t sp = sizeof(T) * (kCartChunk * 3 * (t.p + 1) + kCartChunk * 4);
    k_cart_p2m<T><<<n2, thr, sp, st>>>(b2, n2, D, t.b_begin, t.b_end, t.b_center, t.b_side, t.b_level, t.b_leaf,
                                       t.pos, fs, t.n, M);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_M2M, st);
    const size_t s4 = sizeof(T) * kSets * N;
    for (int l = t.nlevels - 2; l >= 2; --l) {
        const int lb = t.level_off[l], ln = t.level_off[l + 1] - lb;
        if (ln > 0) {
            k_cart_m2m<T><<<ln, thr, s4, st>>>(lb, ln, D, t.b_leaf, t.b_child, t.b_cell, t.b_side, M);
            RPY_LAUNCHED(1);
        }
    }
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_X2L, st);   // the multipole-to-local step
    {
        const int mt = std::max(64, ((D.n_items + kCartItems - 1) / kCartItems + 31) / 32 * 32);
        if (mt > 1024) return RPY_ERR_INTERNAL;
        const size_t sm = s4 + sizeof(T) * size_t(kSets) * D.n_items;
        RPY_TRY(set_cart_smem(k_cart_m2l<T>, sm));
        k_cart_m2l<T><<<n2, mt, sm, st>>>(b2, n2, D, t.v_off, t.v_idx, t.b_cell, t.b_side, t.b_level, M, L);
    }
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_L2L, st);
    for (int l = 3; l < t.nlevels; ++l) {
        const int lb = t.level_off[l], ln = t.level_off[l + 1] - lb;
        if (ln > 0) {
            k_cart_l2l<T><<<ln, thr, s4, st>>>(lb, ln, D, t.b_parent, t.b_cell, t.b_side, L);
            RPY_LAUNCHED(1);
        }
    }
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_STAGE_EVAL, st);
    k_cart_prep<T><<<t.nleaf, thr, s4, st>>>(t.leaves, D, t.b_side, t.b_level, t.b_sys, sc, L, U);
    RPY_LAUNCHED(1);
    k_cart_apply<T><<<int((t.n + 127) / 128), 128, 0, st>>>(t.n, t.bead_leaf, t.leaves, D, t.b_center, t.b_side,
                                                            t.b_level, t.pos, U, ufar);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

template int run_cart_t<double>(Tree &, const double *, double *, const SysConst &, cudaStream_t);
template int run_cart_t<float>(Tree &, const double *, double *, const SysConst &, cudaStream_t);

}  // namespace rpy
