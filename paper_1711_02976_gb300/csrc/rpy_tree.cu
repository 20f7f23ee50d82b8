// Device tree construction: bounding cube, Morton keys, LSD radix sort,
// level-synchronous adaptive octree, colleagues and the U / V / W / X lists
// of the adaptive FMM.
//
// The paper fixes only that the octree is adaptive with a refinement limit
// ("threshold", Sec. 4.2: the maximum number of beads in a childless box).
// Here a box splits while it holds more than leaf_cap beads AND its children
// would still have side >= 2a (so every pair closer than 2a - where the
// Laplace split of Sec. 2 does not hold - stays in the direct near field)
// AND it is above the deepest level.
//
// Lists (adaptive FMM): for a leaf B, U(B) = all leaves adjacent to B
// (including B), W(B) = boxes not adjacent to B whose parent is adjacent to
// B and which descend from a colleague of B; X(B) = {C : B in W(C)};
// V(B) = children of the parent's colleagues that are not adjacent to B.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>

#include "rpy_internal.h"

namespace rpy {

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_err;

void set_last_cuda_error(const char *what, cudaError_t e) {
    g_last_err = std::string(what) + ": " + cudaGetErrorString(e);
}

void set_last_error(const char *msg) { g_last_err = msg; }

int check_cuda(const char *what, cudaError_t e) {
    if (e == cudaSuccess) return RPY_OK;
    set_last_cuda_error(what, e);
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return RPY_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return RPY_ERR_NODEVICE;
    return RPY_ERR_CUDA;
}

const char *last_cuda_error_text() { return g_last_err.c_str(); }

int dev_alloc(Tree &t, void **p, size_t bytes) {
    *p = nullptr;
    Tree &P = t.owner ? *t.owner : t;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    auto it = P.cache.lower_bound(bytes);
    if (it != P.cache.end() && it->first <= 2 * bytes + (size_t(1) << 20)) {
        *p = it->second;
        t.allocs.push_back({it->second, it->first});
        P.cache.erase(it);
        return RPY_OK;
    }
    size_t sz = bytes + bytes / 8;   // slack so that a slightly larger rebuild reuses the block
    cudaError_t e = cudaMalloc(p, sz);
    if (e == cudaErrorMemoryAllocation && !P.cache.empty()) {
        // give the cached blocks back to the device and retry once
        cudaGetLastError();
        for (auto &kv : P.cache) {
            cudaFree(kv.second);
            P.device_bytes -= int64_t(kv.first);
        }
        P.cache.clear();
        e = cudaMalloc(p, sz);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return check_cuda("cudaMalloc", e);
    }
    t.allocs.push_back({*p, sz});
    P.device_bytes += int64_t(sz);
    return RPY_OK;
}

static void dev_free(Tree &t, void *p) {
    if (!p) return;
    Tree &P = t.owner ? *t.owner : t;
    for (size_t i = 0; i < t.allocs.size(); ++i)
        if (t.allocs[i].p == p) {
            P.cache.insert({t.allocs[i].bytes, p});
            t.allocs.erase(t.allocs.begin() + i);
            return;
        }
}

void tree_recycle(Tree &t) {
    Tree &P = t.owner ? *t.owner : t;
    for (auto &b : t.allocs) P.cache.insert({b.bytes, b.p});
    t.allocs.clear();
}

void tree_release(Tree &t) {
    if (t.owner) {
        tree_recycle(t);
        return;
    }
    for (auto &b : t.allocs) cudaFree(b.p);
    for (auto &kv : t.cache) cudaFree(kv.second);
    t.allocs.clear();
    t.cache.clear();
    t.device_bytes = 0;
}

// ---------------------------------------------------------------- scan

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sums[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    int before = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_tile(const int *in, int *out, int n, int *tile_sums) {
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int total;
    int ex = block_exclusive_scan(s, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int *out, int n, const int *tile_off) {
    int base = blockIdx.x * kScanTile;
    int add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

size_t scan_tmp_bytes(int n) {
    size_t b = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        b += 2 * size_t(n) * sizeof(int) + 256;
    }
    return b + 256;
}

static void scan_rec(const int *in, int *out, int n, char *tmp, cudaStream_t st) {
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        RPY_LAUNCHED(1);
        return;
    }
    int *sums = reinterpret_cast<int *>(tmp);
    int *offs = sums + tiles;
    char *next = tmp + ((2 * size_t(tiles) * sizeof(int) + 255) / 256) * 256;
    k_scan_tile<<<tiles, kScanThreads, 0, st>>>(in, out, n, sums);
    RPY_LAUNCHED(1);
    scan_rec(sums, offs, tiles, next, st);
    k_scan_add<<<tiles, kScanThreads, 0, st>>>(out, n, offs);
    RPY_LAUNCHED(1);
}

// *dst = sum of in[0 .. n) after an exclusive scan of it into out (in != out), on the
// device, so that several scans' totals come back in one copy and one synchronisation.
__global__ void k_scan_total(const int *in, const int *out, int n, int *dst) {
    if (threadIdx.x == 0) *dst = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// out[i] = sum_{j<i} in[j]; if total_host, *total_host = sum of all (synchronises st).
int exclusive_scan_i32(const int *in, int *out, int n, int *total_host, void *tmp, size_t tmp_bytes,
                       cudaStream_t st) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return RPY_OK;
    }
    if (tmp_bytes < scan_tmp_bytes(n)) return RPY_ERR_INTERNAL;
    scan_rec(in, out, n, static_cast<char *>(tmp), st);
    RPY_CHECK(cudaGetLastError());
    if (total_host) {
        int a = 0, b = 0;
        RPY_CHECK(cudaMemcpyAsync(&a, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        RPY_CHECK(cudaMemcpyAsync(&b, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        RPY_CHECK(cudaStreamSynchronize(st));
        *total_host = a + b;
    }
    return RPY_OK;
}

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096
constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_radix_hist(const uint64_t *keys, int n, int shift, int *counts, int ntiles) {
    __shared__ int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x)
        if (base + i < n) atomicAdd(&h[(keys[base + i] >> shift) & 255], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: ranks inside the tile follow the input order (warp by warp,
// 32-item rounds in order), tiles are laid out in input order by the scan.  The
// tile is first reordered by digit in shared memory, then written out slot by
// slot, so that consecutive threads store consecutive elements of one digit's run
// (a direct store from the ranking registers sends a warp's 32 stores to up to
// 32 different runs).
constexpr size_t kSortScatterSmem = (sizeof(uint64_t) + sizeof(uint32_t)) * kSortTile;

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t *kin, const uint32_t *vin,
                                                                uint64_t *kout, uint32_t *vout, int n, int shift,
                                                                const int *offs, int ntiles) {
    __shared__ int wh[kSortWarps][257];
    __shared__ int wb[kSortWarps][256];
    __shared__ int tstart[257];   // first slot of each digit in the reordered tile; [256] = valid items
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * 257; i += blockDim.x) (&wh[0][0])[i] = 0;
    __syncthreads();
    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    int rk[kSortItems], dg[kSortItems];
    int base = blockIdx.x * kSortTile + warp * (kSortItems * 32);
    // all of the thread's loads first (independent, so all in flight at once), then the ranking
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int i = base + r * 32 + lane;
        k[r] = i < n ? kin[i] : 0ull;
        v[r] = i < n ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int i = base + r * 32 + lane;
        bool valid = i < n;
        int d = valid ? int((k[r] >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int pre = __popc(peers & ((1u << lane) - 1u));
        int b = 0;
        if (lane == leader) {
            b = wh[warp][d];
            wh[warp][d] = b + __popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        __syncwarp();
        dg[r] = d;
        rk[r] = b + pre;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int s = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            wb[w][d] = s;
            s += wh[w][d];
        }
        tstart[d] = s;   // this tile's count of digit d, scanned below
    }
    __syncthreads();
    {
        const int c = threadIdx.x < 256 ? tstart[threadIdx.x] : 0;
        int total;
        const int ex = block_exclusive_scan(c, &total);
        if (threadIdx.x < 256) tstart[threadIdx.x] = ex;
        if (threadIdx.x == 0) tstart[256] = total;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dg[r] < 256) {
            const int lp = tstart[dg[r]] + wb[warp][dg[r]] + rk[r];
            sk[lp] = k[r];
            sv[lp] = v[r];
        }
    }
    __syncthreads();
    const int nt = tstart[256];
    for (int q = threadIdx.x; q < nt; q += blockDim.x) {
        const uint64_t key = sk[q];
        const int d = int((key >> shift) & 255);
        const int pos = offs[d * ntiles + blockIdx.x] + (q - tstart[d]);
        kout[pos] = key;
        vout[pos] = sv[q];
    }
}

// The scatter's dynamic shared memory (the reordered tile): the limit is raised
// once per device, so that a larger tile may pass the default 48 KB together
// with the static arrays (2,048 items per tile take 24 KB).
static cudaError_t set_scatter_smem() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(dev)) return cudaSuccess;
    e = cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSortScatterSmem));
    if (e == cudaSuccess) done.insert(dev);
    return e;
}

// Sort (keys, vals) by bits [0, bits) stably.  Result ends in (k0, v0).
static int radix_sort(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int n, int bits, int *counts,
                      void *scan_tmp, size_t scan_bytes, cudaStream_t st) {
    RPY_CHECK(set_scatter_smem());
    int ntiles = (n + kSortTile - 1) / kSortTile;
    int passes = (bits + 7) / 8;
    for (int pss = 0; pss < passes; ++pss) {
        int shift = 8 * pss;
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(k0, n, shift, counts, ntiles);
        RPY_LAUNCHED(1);
        RPY_TRY(exclusive_scan_i32(counts, counts, 256 * ntiles, nullptr, scan_tmp, scan_bytes, st));
        k_radix_scatter<<<ntiles, kSortThreads, kSortScatterSmem, st>>>(k0, v0, k1, v1, n, shift, counts, ntiles);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    if (passes & 1) {   // result is in the second buffer: copy back
        RPY_CHECK(cudaMemcpyAsync(k1, k0, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        RPY_CHECK(cudaMemcpyAsync(v1, v0, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return RPY_OK;
}

// ---------------------------------------------------------------- cube, keys

constexpr int kChunk = 8192;

// chunk c covers beads [cb[c], ce[c]) of system cs[c]
__global__ void k_bbox_partial(const double *pos, const int64_t *cb, const int64_t *ce, double *part,
                               unsigned *status) {
    __shared__ double red[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = cb[blockIdx.x] + threadIdx.x; i < ce[blockIdx.x]; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double v = pos[3 * i + a];
            if (!isfinite(v)) bad = true;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    if (bad) atomicOr(status, DEVERR_NONFINITE);
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = lo[a];
        red[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + s]);
                red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// cube of system s (one block per system): the chunk partials folded by min / max
// (exact, so the order does not matter), then centre = (lo+hi)/2, side = max extent
// (exact IEEE ops, no contraction).  kq[s] = the key grid's origin per axis,
// origin = centre - side/2, and RN(1/side) * 2^21 (= RN(2^21/side): the power of two
// scales exactly), for k_morton.
constexpr int kBoxFinalThreads = 128;
__global__ void k_bbox_final(const double *part, const int *sys_chunk_off, double *cube, double *kq) {
    __shared__ double red[6][kBoxFinalThreads];
    const int s = blockIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = sys_chunk_off[s] + threadIdx.x; c < sys_chunk_off[s + 1]; c += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], part[6 * c + a]);
            hi[a] = fmax(hi[a], part[6 * c + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = lo[a];
        red[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + h]);
                red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + h]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double side = 0.0;
        for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(red[3 + a][0], red[a][0]));
        for (int a = 0; a < 3; ++a) {
            const double c = __dmul_rn(0.5, __dadd_rn(red[a][0], red[3 + a][0]));
            cube[4 * s + a] = c;
            kq[4 * s + a] = __dsub_rn(c, __dmul_rn(0.5, side));
        }
        cube[4 * s + 3] = side;
        kq[4 * s + 3] = side == 0.0 ? 0.0 : __dmul_rn(__drcp_rn(side), 2097152.0);
    }
}

__device__ __forceinline__ int sys_of(const int64_t *off, int nsys, int64_t i) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// q = min(2^21-1, floor((x - origin)/side * 2^21)), origin = centre - side/2,
// every step a single correctly rounded operation (no FMA contraction).
// The scaled quotient is formed as d * RN(2^21/side): two roundings instead of
// one put it within 3.5e-16 (relative, for |d| <= side) of RN(d / side) * 2^21,
// i.e. within 7.3e-10 of it, so its floor is that of the defined value unless
// it lies within 1e-9 of an integer; there the correctly rounded division is
// taken.  The band test compares the bit patterns of the fraction (non-negative
// doubles order as integers), and the integer is read from the mantissa after
// adding 2^52 (exact for integers below 2^52): no FP64 conversions.
__global__ void k_morton(const double *pos, int64_t n, const int64_t *off, int nsys, const double *cube,
                         const double *kq, uint64_t *keys, uint64_t *keys_copy, uint32_t *idx, uint64_t *sysk) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = sys_of(off, nsys, i);
    const double inv21 = kq[4 * s + 3];
    const long long lo_band = __double_as_longlong(1e-9), hi_band = __double_as_longlong(1.0 - 1e-9);
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        if (inv21 == 0.0) {   // side 0: every bead at the centre
            q[a] = 0;
            continue;
        }
        const double d = __dsub_rn(pos[3 * i + a], kq[4 * s + a]);
        const double t2 = __dmul_rn(d, inv21);
        double fl = floor(t2);
        const long long fr = __double_as_longlong(__dsub_rn(t2, fl));   // fraction in [0, 1), exact
        if (fr < lo_band || fr > hi_band) fl = floor(__dmul_rn(__ddiv_rn(d, cube[4 * s + 3]), 2097152.0));
        fl = fl < 0.0 ? 0.0 : fl;
        fl = fl > 2097151.0 ? 2097151.0 : fl;
        q[a] = uint64_t(__double_as_longlong(__dadd_rn(fl, 4503599627370496.0))) & 0x1fffffull;
    }
    uint64_t key = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    keys[i] = key;
    keys_copy[i] = key;
    idx[i] = uint32_t(i);
    if (sysk) sysk[i] = uint64_t(s);
}

// keys_sorted: the keys already in sorted order (one system: the sort's own output),
// read in place of the gather from keys_caller
__global__ void k_gather_sorted(const double *pos, int64_t n, const uint32_t *perm, const uint64_t *keys_caller,
                                const uint64_t *keys_sorted, const int64_t *off, int nsys, double *pos_s,
                                uint64_t *keys_s, int *perm_i, int *bead_sys) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = perm[i];
    pos_s[i] = pos[3 * int64_t(j)];
    pos_s[n + i] = pos[3 * int64_t(j) + 1];
    pos_s[2 * n + i] = pos[3 * int64_t(j) + 2];
    keys_s[i] = keys_sorted ? keys_sorted[i] : keys_caller[j];
    perm_i[i] = int(j);
    bead_sys[i] = sys_of(off, nsys, int64_t(j));
}

__global__ void k_sysk_from_perm(const uint32_t *vals, int64_t n, const int64_t *off, int nsys, uint64_t *sysk) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sysk[i] = uint64_t(sys_of(off, nsys, int64_t(vals[i])));
}

// ---------------------------------------------------------------- octree

__global__ void k_roots(int nsys, const int64_t *off, const double *cube, int *lvl, int *beg, int *end, int *par,
                        int *child, int *coll, int *cell, int *bsys, int *leaf, double *ctr, double *side) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    lvl[s] = 0;
    beg[s] = int(off[s]);
    end[s] = int(off[s + 1]);
    par[s] = -1;
    for (int o = 0; o < 8; ++o) child[8 * s + o] = -1;
    for (int q = 0; q < 27; ++q) coll[27 * s + q] = -1;
    coll[27 * s + 13] = s;
    for (int a = 0; a < 3; ++a) {
        cell[3 * s + a] = 0;
        ctr[3 * s + a] = cube[4 * s + a];
    }
    side[s] = cube[4 * s + 3];
    bsys[s] = s;
    leaf[s] = 1;
}

__global__ void k_split_count(int b0, int nb, int level, int cap, int max_level, const int *beg, const int *end,
                              const double *side, const int *bsys, const double *sys_a, const uint64_t *keys,
                              int *bounds, int *nchild) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nb) return;
    if (i == nb) { nchild[i] = 0; return; }
    int b = b0 + i;
    int lo = beg[b], hi = end[b];
    double a = sys_a[bsys[b]];
    bool split = (hi - lo) > cap && 0.5 * side[b] >= 2.0 * a && level < max_level;
    int cnt = 0;
    if (split) {
        int sh = 60 - 3 * level;
        bounds[9 * i] = lo;
        for (int o = 1; o < 8; ++o) {
            int l = lo, h = hi;   // first index with digit >= o
            while (l < h) {
                int mid = (l + h) >> 1;
                if (int((keys[mid] >> sh) & 7ull) < o) l = mid + 1; else h = mid;
            }
            bounds[9 * i + o] = l;
        }
        bounds[9 * i + 8] = hi;
        for (int o = 0; o < 8; ++o) cnt += bounds[9 * i + o + 1] > bounds[9 * i + o];
    }
    nchild[i] = cnt;
}

__global__ void k_make_children(int b0, int nb, int level, int first_new, const int *bounds, const int *nchild,
                                const int *cbase, int *lvl, int *beg, int *end, int *par, int *child, int *coll,
                                int *cell, int *bsys, int *leaf, double *ctr, double *side) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int b = b0 + i;
    if (nchild[i] == 0) return;
    leaf[b] = 0;
    int c = first_new + cbase[i];
    double hs = 0.5 * side[b];
    for (int o = 0; o < 8; ++o) {
        int lo = bounds[9 * i + o], hi = bounds[9 * i + o + 1];
        if (hi <= lo) { child[8 * b + o] = -1; continue; }
        child[8 * b + o] = c;
        lvl[c] = level + 1;
        beg[c] = lo;
        end[c] = hi;
        par[c] = b;
        for (int k = 0; k < 8; ++k) child[8 * c + k] = -1;
        for (int q = 0; q < 27; ++q) coll[27 * c + q] = -1;
        for (int a = 0; a < 3; ++a) {
            int bit = (o >> a) & 1;
            cell[3 * c + a] = 2 * cell[3 * b + a] + bit;
            ctr[3 * c + a] = ctr[3 * b + a] + (bit ? 0.5 : -0.5) * hs;
        }
        side[c] = hs;
        bsys[c] = bsys[b];
        leaf[c] = 1;
        ++c;
    }
}

__device__ __forceinline__ bool boxes_adjacent(int la, const int *ca, int lb, const int *cb) {
    // closed boxes touch or overlap
    if (la > lb) {
        int t = la; la = lb; lb = t;
        const int *tc = ca; ca = cb; cb = tc;
    }
    int sh = lb - la;
    for (int a = 0; a < 3; ++a) {
        long lo = long(ca[a]) << sh, hi = long(ca[a] + 1) << sh;
        if (long(cb[a]) + 1 < lo || long(cb[a]) > hi) return false;
    }
    return true;
}

__global__ void k_colleagues(int b0, int nb, const int *par, const int *child, int *coll, const int *cell) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int b = b0 + i;
    int p = par[b];
    for (int q = 0; q < 27; ++q) {
        int Q = coll[27 * p + q];
        if (Q < 0) continue;
        for (int o = 0; o < 8; ++o) {
            int c = child[8 * Q + o];
            if (c < 0) continue;
            int d[3];
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                d[a] = cell[3 * c + a] - cell[3 * b + a];
                if (d[a] < -1 || d[a] > 1) ok = false;
            }
            if (ok) coll[27 * b + (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1)] = c;
        }
    }
}

// ---------------------------------------------------------------- lists

struct ListArgs {
    const int *lvl, *par, *child, *coll, *cell, *leaf, *leafid, *beg, *end;
    int tw, tx;                          // direct-substitution thresholds (0 = none)
    int *ucnt, *wcnt, *xcnt, *wdcnt, *xdcnt;            // count pass
    const int *uoff, *woff, *xoff, *wdoff, *xdoff;      // fill pass
    int *uidx, *widx, *xidx, *wdidx, *xdidx;
    unsigned *status;
};

constexpr int kStack = 96;

__device__ __forceinline__ int box_count(const ListArgs &A, int b) { return A.end[b] - A.beg[b]; }

template <bool FILL>
__global__ void k_lists(int nbox, ListArgs A) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int lb = A.lvl[b];
    const int *cb = A.cell + 3 * b;
    // X list: leaf colleagues of ancestors, adjacent to the parent, not to b.
    // Small target boxes take their X sources directly (XD).
    bool xdirect = A.tx > 0 && box_count(A, b) <= A.tx;
    int nx = 0, xo = 0;
    if (FILL) xo = xdirect ? A.xdoff[b] : A.xoff[b];
    int P = A.par[b];
    if (P >= 0) {
        for (int anc = P; anc >= 0; anc = A.par[anc]) {
            for (int q = 0; q < 27; ++q) {
                int c = A.coll[27 * anc + q];
                if (c < 0 || c == anc || !A.leaf[c]) continue;
                int lc = A.lvl[c];
                if (boxes_adjacent(lc, A.cell + 3 * c, lb, cb)) continue;
                if (!boxes_adjacent(lc, A.cell + 3 * c, A.lvl[P], A.cell + 3 * P)) continue;
                if (FILL) (xdirect ? A.xdidx : A.xidx)[xo + nx] = c;
                ++nx;
            }
        }
    }
    if (!FILL) {
        A.xcnt[b] = xdirect ? 0 : nx;
        A.xdcnt[b] = xdirect ? nx : 0;
    }
    if (!A.leaf[b]) return;
    int li = A.leafid[b];
    int nu = 0, nw = 0, nwd = 0;
    int uo = FILL ? A.uoff[li] : 0, wo = FILL ? A.woff[li] : 0, wdo = FILL ? A.wdoff[li] : 0;
    // (a) same-level leaf colleagues, b included
    for (int q = 0; q < 27; ++q) {
        int c = A.coll[27 * b + q];
        if (c >= 0 && A.leaf[c]) {
            if (FILL) A.uidx[uo + nu] = c;
            ++nu;
        }
    }
    // (b) coarser leaves adjacent to b: leaf colleagues of ancestors
    for (int anc = P; anc >= 0; anc = A.par[anc]) {
        for (int q = 0; q < 27; ++q) {
            int c = A.coll[27 * anc + q];
            if (c < 0 || c == anc || !A.leaf[c]) continue;
            if (!boxes_adjacent(A.lvl[c], A.cell + 3 * c, lb, cb)) continue;
            if (FILL) A.uidx[uo + nu] = c;
            ++nu;
        }
    }
    // (c) finer: descend into non-leaf colleagues; non-adjacent children form W
    int stack[kStack];
    int sp = 0;
    for (int q = 0; q < 27; ++q) {
        int c = A.coll[27 * b + q];
        if (c >= 0 && !A.leaf[c]) stack[sp++] = c;
    }
    while (sp > 0) {
        int c = stack[--sp];
        for (int o = 0; o < 8; ++o) {
            int ch = A.child[8 * c + o];
            if (ch < 0) continue;
            if (boxes_adjacent(A.lvl[ch], A.cell + 3 * ch, lb, cb)) {
                if (A.leaf[ch]) {
                    if (FILL) A.uidx[uo + nu] = ch;
                    ++nu;
                } else if (sp < kStack) {
                    stack[sp++] = ch;
                } else {
                    atomicOr(A.status, DEVERR_STACK);
                }
            } else if (A.tw > 0 && box_count(A, ch) <= A.tw) {
                if (FILL) A.wdidx[wdo + nwd] = ch;
                ++nwd;
            } else {
                if (FILL) A.widx[wo + nw] = ch;
                ++nw;
            }
        }
    }
    if (!FILL) {
        A.ucnt[li] = nu;
        A.wcnt[li] = nw;
        A.wdcnt[li] = nwd;
    }
}

// Direct list of leaf b: its direct W sources, then the direct X sources of b
// and of every ancestor whose X sources are taken directly (those are exactly
// the ancestors holding at most tx beads, a chain upward from b).
template <bool FILL>
__global__ void k_dlists(int nleaf, const int *leaves, const int *par, const int *beg, const int *end, int tx,
                         const int *wdoff, const int *wdidx, const int *xdoff, const int *xdidx, int *dcnt,
                         const int *doff, int *didx) {
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    int b = leaves[li];
    int nd = 0, o = FILL ? doff[li] : 0;
    for (int k = wdoff[li]; k < wdoff[li + 1]; ++k) {
        if (FILL) didx[o + nd] = wdidx[k];
        ++nd;
    }
    if (tx > 0)
        for (int a = b; a >= 0 && end[a] - beg[a] <= tx; a = par[a])
            for (int k = xdoff[a]; k < xdoff[a + 1]; ++k) {
                if (FILL) didx[o + nd] = xdidx[k];
                ++nd;
            }
    if (!FILL) dcnt[li] = nd;
}

template <bool FILL>
__global__ void k_vlists(int b0, int nbox, const int *lvl, const int *par, const int *child, const int *coll,
                         const int *cell, const int *leaf, int *vcnt, const int *voff, int *vidx) {
    int b = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int P = par[b];
    int nv = 0, vo = FILL ? voff[b] : 0;
    if (P >= 0 && lvl[b] >= 2) {
        for (int q = 0; q < 27; ++q) {
            int Q = coll[27 * P + q];
            if (Q < 0 || leaf[Q]) continue;
            for (int o = 0; o < 8; ++o) {
                int c = child[8 * Q + o];
                if (c < 0) continue;
                if (boxes_adjacent(lvl[c], cell + 3 * c, lvl[b], cell + 3 * b)) continue;
                if (FILL) vidx[vo + nv] = c;
                ++nv;
            }
        }
    }
    if (!FILL) vcnt[b] = nv;
}

__global__ void k_flag_compact(int n, const int *flag, const int *pos, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = i;
}

__global__ void k_leafid(int n, const int *leaf, const int *pos, int *leafid) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) leafid[i] = leaf[i] ? pos[i] : -1;
}

__global__ void k_bead_leaf(int nleaf, const int *leaves, const int *beg, const int *end, int *bead_leaf) {
    int li = blockIdx.x;
    if (li >= nleaf) return;
    int b = leaves[li];
    for (int i = beg[b] + threadIdx.x; i < end[b]; i += blockDim.x) bead_leaf[i] = li;
}

__global__ void k_x2x_flag(int b0, int nbox, const int *leaf, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbox) flag[i] = (i >= b0 && !leaf[i]) ? 1 : 0;
}

__global__ void k_leaf_stats(int nleaf, const int *leaves, const int *beg, const int *end, const int *uoff,
                             const int *uidx, const int *doff, const int *didx, int cap, unsigned long long *pairs,
                             int *maxcnt, int *over) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long ps = 0, pd = 0;   // this leaf's U-list and direct pairs
    int nb = 0, ov = 0;
    if (i < nleaf) {
        int b = leaves[i];
        nb = end[b] - beg[b];
        unsigned long long s = 0, sd = 0;
        for (int k = uoff[i]; k < uoff[i + 1]; ++k) s += unsigned(end[uidx[k]] - beg[uidx[k]]);
        for (int k = doff[i]; k < doff[i + 1]; ++k) sd += unsigned(end[didx[k]] - beg[didx[k]]);
        ps = s * unsigned(nb);
        pd = sd * unsigned(nb);
        ov = nb > cap;
    }
    // integer sums and maximum over the warp, then one atomic of each per warp (one per
    // leaf on a single word serialised on the hundreds of thousands of leaves of a forest)
    for (int o = 16; o > 0; o >>= 1) {
        ps += __shfl_down_sync(0xffffffffu, ps, o);
        pd += __shfl_down_sync(0xffffffffu, pd, o);
        nb = max(nb, __shfl_down_sync(0xffffffffu, nb, o));
        ov += __shfl_down_sync(0xffffffffu, ov, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ps) atomicAdd(pairs, ps);
        if (pd) atomicAdd(pairs + 1, pd);
        atomicMax(maxcnt, nb);
        if (ov) atomicAdd(over, ov);
    }
}

// ---------------------------------------------------------------- near-field work items
// One item per (leaf, block of up to kItemTargets targets).  Two orders list the
// items by decreasing cost, targets x sources in powers of two (one radix pass),
// for the U-list pass and for the direct-substitute pass: the block scheduler
// then starts the long items first, and a leaf that the 2a rule left large is
// spread over several CTAs instead of running alone at the end of the launch.
__global__ void k_item_count(int nleaf, const int *leaves, const int *beg, const int *end, int *cnt) {
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li > nleaf) return;
    if (li == nleaf) {
        cnt[li] = 0;
        return;
    }
    int b = leaves[li];
    cnt[li] = (end[b] - beg[b] + kItemTargets - 1) / kItemTargets;
}

__device__ __forceinline__ uint64_t cost_key(unsigned long long c) {
    return uint64_t(63 - (c ? 63 - __clzll(c) : 0));   // larger cost, smaller key
}

__global__ void k_item_fill(int nleaf, const int *leaves, const int *beg, const int *end, const int *uoff,
                            const int *uidx, const int *doff, const int *didx, const int *ioff, int2 *items,
                            uint64_t *ku, uint32_t *vu, uint64_t *kd, uint32_t *vd, uint64_t *km, uint32_t *vm) {
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    int b = leaves[li];
    int t0 = beg[b], nt = end[b] - t0;
    unsigned long long su = 0, sd = 0;
    for (int k = uoff[li]; k < uoff[li + 1]; ++k) su += unsigned(end[uidx[k]] - beg[uidx[k]]);
    for (int k = doff[li]; k < doff[li + 1]; ++k) sd += unsigned(end[didx[k]] - beg[didx[k]]);
    for (int q = 0, it = ioff[li]; q * kItemTargets < nt; ++q, ++it) {
        unsigned tc = unsigned(min(kItemTargets, nt - q * kItemTargets));
        items[it] = make_int2(li, t0 + q * kItemTargets);
        ku[it] = cost_key(su * tc);
        vu[it] = uint32_t(it);
        kd[it] = cost_key(sd * tc);
        vd[it] = uint32_t(it);
        km[it] = cost_key((su + sd) * tc);
        vm[it] = uint32_t(it);
    }
}

__global__ void k_item_order(int n, const int2 *items, const uint32_t *ou, const uint32_t *od, const uint32_t *om,
                             int2 *u_items, int2 *d_items, int2 *m_items) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u_items[i] = items[ou[i]];
    d_items[i] = items[od[i]];
    m_items[i] = items[om[i]];
}

// The near list of the full matvec: per leaf its U list followed by its direct
// substitutes (m_off = u_off + d_off, both exclusive prefix sums over leaves).
__global__ void k_merge_lists(int nleaf, const int *uoff, const int *uidx, const int *doff, const int *didx,
                              int *moff, int *midx) {
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li > nleaf) return;
    const int m0 = uoff[li] + doff[li];
    moff[li] = m0;
    if (li == nleaf) return;
    int q = m0;
    for (int k = uoff[li]; k < uoff[li + 1]; ++k) midx[q++] = uidx[k];
    for (int k = doff[li]; k < doff[li + 1]; ++k) midx[q++] = didx[k];
}

// ---------------------------------------------------------------- build driver

static int grow_boxes(Tree &t, int need, cudaStream_t st) {
    if (need <= t.nbox_cap) return RPY_OK;
    int cap = std::max(need, t.nbox_cap * 2);
    cap = std::max(cap, 1024);
    struct F { void **p; size_t es; int per; };
    F fields[] = {{(void **)&t.b_level, 4, 1}, {(void **)&t.b_begin, 4, 1}, {(void **)&t.b_end, 4, 1},
                  {(void **)&t.b_parent, 4, 1}, {(void **)&t.b_child, 4, 8}, {(void **)&t.b_coll, 4, 27},
                  {(void **)&t.b_cell, 4, 3}, {(void **)&t.b_sys, 4, 1}, {(void **)&t.b_leaf, 4, 1},
                  {(void **)&t.b_center, 8, 3}, {(void **)&t.b_side, 8, 1}};
    for (auto &f : fields) {
        void *np = nullptr;
        RPY_TRY(dev_alloc(t, &np, f.es * f.per * size_t(cap)));
        if (*f.p) {
            RPY_CHECK(cudaMemcpyAsync(np, *f.p, f.es * f.per * size_t(t.nbox), cudaMemcpyDeviceToDevice, st));
            dev_free(t, *f.p);
        }
        *f.p = np;
    }
    t.nbox_cap = cap;
    return RPY_OK;
}

static inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

int tree_build(Tree &t, const double *pos_dev, cudaStream_t st) {
    const int64_t n = t.n;
    const int nsys = t.nsys;
    // -- per-system chunk table for the bounding cubes
    std::vector<int64_t> cb, ce;
    std::vector<int> sco(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        sco[s] = int(cb.size());
        for (int64_t i = t.sys_off_h[s]; i < t.sys_off_h[s + 1]; i += kChunk) {
            cb.push_back(i);
            ce.push_back(std::min(i + kChunk, t.sys_off_h[s + 1]));
        }
    }
    sco[nsys] = int(cb.size());
    int nch = int(cb.size());
    // scratch for the build (returned to the tree's block cache at the end, and
    // on every early return)
    Tree scratch;
    scratch.owner = &t;
    struct ScratchGuard {
        Tree &s;
        ~ScratchGuard() { tree_release(s); }
    } scratch_guard{scratch};
    int64_t *d_cb, *d_ce;
    int *d_sco;
    double *d_part;
    RPY_TRY(dev_alloc(scratch, (void **)&d_cb, sizeof(int64_t) * nch));
    RPY_TRY(dev_alloc(scratch, (void **)&d_ce, sizeof(int64_t) * nch));
    RPY_TRY(dev_alloc(scratch, (void **)&d_sco, sizeof(int) * (nsys + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&d_part, sizeof(double) * 6 * nch));
    RPY_CHECK(cudaMemcpyAsync(d_cb, cb.data(), sizeof(int64_t) * nch, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(d_ce, ce.data(), sizeof(int64_t) * nch, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(d_sco, sco.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemsetAsync(t.dev_status, 0, sizeof(unsigned), st));
    k_bbox_partial<<<nch, 256, 0, st>>>(pos_dev, d_cb, d_ce, d_part, t.dev_status);
    RPY_LAUNCHED(1);
    double *d_kq;
    RPY_TRY(dev_alloc(scratch, (void **)&d_kq, sizeof(double) * 4 * nsys));
    k_bbox_final<<<nsys, kBoxFinalThreads, 0, st>>>(d_part, d_sco, t.sys_cube, d_kq);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    unsigned status = 0;
    RPY_CHECK(cudaMemcpyAsync(&status, t.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    if (status & DEVERR_NONFINITE) {
        tree_release(scratch);
        return RPY_ERR_NONFINITE;
    }
    // -- keys and sort
    uint64_t *k0, *k1, *kcaller, *sysk = nullptr;
    uint32_t *v0, *v1;
    RPY_TRY(dev_alloc(scratch, (void **)&k0, sizeof(uint64_t) * n));
    RPY_TRY(dev_alloc(scratch, (void **)&k1, sizeof(uint64_t) * n));
    RPY_TRY(dev_alloc(scratch, (void **)&kcaller, sizeof(uint64_t) * n));
    RPY_TRY(dev_alloc(scratch, (void **)&v0, sizeof(uint32_t) * n));
    RPY_TRY(dev_alloc(scratch, (void **)&v1, sizeof(uint32_t) * n));
    int ntiles = nblk(n, kSortTile);
    int *counts;
    RPY_TRY(dev_alloc(scratch, (void **)&counts, sizeof(int) * 256 * size_t(ntiles)));
    size_t sbytes = std::max(scan_tmp_bytes(256 * ntiles), scan_tmp_bytes(int(n) + 1));
    void *stmp;
    RPY_TRY(dev_alloc(scratch, &stmp, sbytes));
    if (nsys > 1) RPY_TRY(dev_alloc(scratch, (void **)&sysk, sizeof(uint64_t) * n));
    k_morton<<<nblk(n, 256), 256, 0, st>>>(pos_dev, n, t.sys_off, nsys, t.sys_cube, d_kq, k0, kcaller, v0, nullptr);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_TRY(radix_sort(k0, v0, k1, v1, int(n), 63, counts, stmp, sbytes, st));
    if (nsys > 1) {
        k_sysk_from_perm<<<nblk(n, 256), 256, 0, st>>>(v0, n, t.sys_off, nsys, sysk);
        RPY_LAUNCHED(1);
        int bits = 1;
        while ((1 << bits) < nsys) ++bits;
        RPY_TRY(radix_sort(sysk, v0, k1, v1, int(n), bits, counts, stmp, sbytes, st));
    }
    k_gather_sorted<<<nblk(n, 256), 256, 0, st>>>(pos_dev, n, v0, kcaller, nsys == 1 ? k0 : nullptr, t.sys_off, nsys,
                                                  t.pos, t.keys, t.perm, t.bead_sys);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    // -- octree, level by level
    t.nbox = 0;
    RPY_TRY(grow_boxes(t, std::max(nsys * 64, int(std::min<int64_t>(n, 1 << 20) / 4 + 64)), st));
    k_roots<<<nblk(nsys, 128), 128, 0, st>>>(nsys, t.sys_off, t.sys_cube, t.b_level, t.b_begin, t.b_end,
                                             t.b_parent, t.b_child, t.b_coll, t.b_cell, t.b_sys, t.b_leaf,
                                             t.b_center, t.b_side);
    RPY_LAUNCHED(1);
    t.nbox = nsys;
    t.level_off.assign(1, 0);
    t.level_off.push_back(nsys);
    int maxl = t.params.max_level;
    int *bounds = nullptr, *nchild = nullptr, *cbase = nullptr;
    int bcap = 0;
    for (int level = 0;; ++level) {
        int b0 = t.level_off[level], nb = t.level_off[level + 1] - b0;
        if (nb == 0) break;
        if (nb + 1 > bcap) {
            if (bounds) { dev_free(scratch, bounds); dev_free(scratch, nchild); dev_free(scratch, cbase); }
            bcap = std::max(2 * (nb + 1), 4096);
            RPY_TRY(dev_alloc(scratch, (void **)&bounds, sizeof(int) * 9 * size_t(bcap)));
            RPY_TRY(dev_alloc(scratch, (void **)&nchild, sizeof(int) * size_t(bcap)));
            RPY_TRY(dev_alloc(scratch, (void **)&cbase, sizeof(int) * size_t(bcap)));
        }
        k_split_count<<<nblk(nb + 1, 256), 256, 0, st>>>(b0, nb, level, t.params.leaf_cap, maxl, t.b_begin, t.b_end,
                                                         t.b_side, t.b_sys, t.sys_a, t.keys, bounds, nchild);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
        int total = 0;
        if (scan_tmp_bytes(nb + 1) > sbytes) return RPY_ERR_INTERNAL;
        RPY_TRY(exclusive_scan_i32(nchild, cbase, nb + 1, &total, stmp, sbytes, st));
        if (total == 0) break;
        RPY_TRY(grow_boxes(t, t.nbox + total, st));
        k_make_children<<<nblk(nb, 256), 256, 0, st>>>(b0, nb, level, t.nbox, bounds, nchild, cbase, t.b_level,
                                                       t.b_begin, t.b_end, t.b_parent, t.b_child, t.b_coll,
                                                       t.b_cell, t.b_sys, t.b_leaf, t.b_center, t.b_side);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
        t.nbox += total;
        t.level_off.push_back(t.nbox);
    }
    t.nlevels = int(t.level_off.size()) - 1;
    // -- colleagues
    for (int level = 1; level < t.nlevels; ++level) {
        int b0 = t.level_off[level], nb = t.level_off[level + 1] - b0;
        k_colleagues<<<nblk(nb, 128), 128, 0, st>>>(b0, nb, t.b_parent, t.b_child, t.b_coll, t.b_cell);
        RPY_LAUNCHED(1);
    }
    RPY_CHECK(cudaGetLastError());
    // -- leaves
    int nbx = t.nbox;
    if (scan_tmp_bytes(nbx + 1) > sbytes) {
        dev_free(scratch, stmp);
        sbytes = scan_tmp_bytes(nbx + 1) + 4096;
        RPY_TRY(dev_alloc(scratch, &stmp, sbytes));
    }
    int *pos_tmp;
    RPY_TRY(dev_alloc(scratch, (void **)&pos_tmp, sizeof(int) * (nbx + 1)));
    int nleaf = 0;
    RPY_TRY(exclusive_scan_i32(t.b_leaf, pos_tmp, nbx, &nleaf, stmp, sbytes, st));
    t.nleaf = nleaf;
    RPY_TRY(dev_alloc(t, (void **)&t.leaves, sizeof(int) * nleaf));
    RPY_TRY(dev_alloc(t, (void **)&t.b_leafid, sizeof(int) * nbx));
    k_flag_compact<<<nblk(nbx, 256), 256, 0, st>>>(nbx, t.b_leaf, pos_tmp, t.leaves);
    RPY_LAUNCHED(1);
    k_leafid<<<nblk(nbx, 256), 256, 0, st>>>(nbx, t.b_leaf, pos_tmp, t.b_leafid);
    RPY_LAUNCHED(1);
    RPY_TRY(dev_alloc(t, (void **)&t.bead_leaf, sizeof(int) * n));
    if (nleaf > 0) {
        k_bead_leaf<<<nleaf, 64, 0, st>>>(nleaf, t.leaves, t.b_begin, t.b_end, t.bead_leaf);
        RPY_LAUNCHED(1);
    }
    // -- X2X parents: non-leaf boxes at level >= 1
    {
        int *flag;
        RPY_TRY(dev_alloc(scratch, (void **)&flag, sizeof(int) * (nbx + 1)));
        int b0 = t.nlevels > 1 ? t.level_off[1] : nbx;
        k_x2x_flag<<<nblk(nbx, 256), 256, 0, st>>>(b0, nbx, t.b_leaf, flag);
        RPY_LAUNCHED(1);
        int np = 0;
        RPY_TRY(exclusive_scan_i32(flag, pos_tmp, nbx, &np, stmp, sbytes, st));
        t.n_x2x_par = np;
        RPY_TRY(dev_alloc(t, (void **)&t.x2x_par, sizeof(int) * std::max(np, 1)));
        k_flag_compact<<<nblk(nbx, 256), 256, 0, st>>>(nbx, flag, pos_tmp, t.x2x_par);
        RPY_LAUNCHED(1);
    }
    // -- lists
    ListArgs A{};
    A.lvl = t.b_level; A.par = t.b_parent; A.child = t.b_child; A.coll = t.b_coll; A.cell = t.b_cell;
    A.leaf = t.b_leaf; A.leafid = t.b_leafid; A.beg = t.b_begin; A.end = t.b_end; A.status = t.dev_status;
    A.tw = t.direct_w; A.tx = t.direct_x;
    int *ucnt, *wcnt, *xcnt, *wdcnt, *xdcnt, *wdoff, *xdoff, *wdidx, *xdidx, *dcnt;
    RPY_TRY(dev_alloc(scratch, (void **)&ucnt, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&wcnt, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&wdcnt, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&dcnt, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&xcnt, sizeof(int) * (nbx + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&xdcnt, sizeof(int) * (nbx + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&wdoff, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&xdoff, sizeof(int) * (nbx + 1)));
    for (int *z : {ucnt, wcnt, wdcnt, dcnt})
        RPY_CHECK(cudaMemsetAsync(z, 0, sizeof(int) * (nleaf + 1), st));
    for (int *z : {xcnt, xdcnt}) RPY_CHECK(cudaMemsetAsync(z, 0, sizeof(int) * (nbx + 1), st));
    A.ucnt = ucnt; A.wcnt = wcnt; A.xcnt = xcnt; A.wdcnt = wdcnt; A.xdcnt = xdcnt;
    k_lists<false><<<nblk(nbx, 128), 128, 0, st>>>(nbx, A);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_TRY(dev_alloc(t, (void **)&t.u_off, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.w_off, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.x_off, sizeof(int) * (nbx + 1)));
    // the five list offsets: scans in stream order, their totals read back together
    int tot[5] = {0, 0, 0, 0, 0};
    {
        int *dtot;
        RPY_TRY(dev_alloc(scratch, (void **)&dtot, sizeof(tot)));
        const int *sin[5] = {ucnt, wcnt, xcnt, wdcnt, xdcnt};
        int *sout[5] = {t.u_off, t.w_off, t.x_off, wdoff, xdoff};
        const int sn[5] = {nleaf + 1, nleaf + 1, nbx + 1, nleaf + 1, nbx + 1};
        for (int j = 0; j < 5; ++j) {
            RPY_TRY(exclusive_scan_i32(sin[j], sout[j], sn[j], nullptr, stmp, sbytes, st));
            k_scan_total<<<1, 32, 0, st>>>(sin[j], sout[j], sn[j], dtot + j);
            RPY_LAUNCHED(1);
        }
        RPY_CHECK(cudaGetLastError());
        RPY_CHECK(cudaMemcpyAsync(tot, dtot, sizeof(tot), cudaMemcpyDeviceToHost, st));
        RPY_CHECK(cudaStreamSynchronize(st));
    }
    const int nu = tot[0], nw = tot[1], nx = tot[2], nwd = tot[3], nxd = tot[4];
    t.n_u = nu; t.n_w = nw; t.n_x = nx;
    RPY_TRY(dev_alloc(t, (void **)&t.u_idx, sizeof(int) * std::max(nu, 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.w_idx, sizeof(int) * std::max(nw, 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.x_idx, sizeof(int) * std::max(nx, 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&wdidx, sizeof(int) * std::max(nwd, 1)));
    RPY_TRY(dev_alloc(scratch, (void **)&xdidx, sizeof(int) * std::max(nxd, 1)));
    A.uoff = t.u_off; A.woff = t.w_off; A.xoff = t.x_off; A.wdoff = wdoff; A.xdoff = xdoff;
    A.uidx = t.u_idx; A.widx = t.w_idx; A.xidx = t.x_idx; A.wdidx = wdidx; A.xdidx = xdidx;
    k_lists<true><<<nblk(nbx, 128), 128, 0, st>>>(nbx, A);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    // per-leaf direct lists
    k_dlists<false><<<nblk(nleaf, 128), 128, 0, st>>>(nleaf, t.leaves, t.b_parent, t.b_begin, t.b_end, t.direct_x,
                                                      wdoff, wdidx, xdoff, xdidx, dcnt, nullptr, nullptr);
    RPY_LAUNCHED(1);
    RPY_TRY(dev_alloc(t, (void **)&t.d_off, sizeof(int) * (nleaf + 1)));
    int nd = 0;
    RPY_TRY(exclusive_scan_i32(dcnt, t.d_off, nleaf + 1, &nd, stmp, sbytes, st));
    t.n_d = nd;
    RPY_TRY(dev_alloc(t, (void **)&t.d_idx, sizeof(int) * std::max(nd, 1)));
    k_dlists<true><<<nblk(nleaf, 128), 128, 0, st>>>(nleaf, t.leaves, t.b_parent, t.b_begin, t.b_end, t.direct_x,
                                                     wdoff, wdidx, xdoff, xdidx, nullptr, t.d_off, t.d_idx);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_TRY(dev_alloc(t, (void **)&t.m_off, sizeof(int) * (nleaf + 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.m_idx, sizeof(int) * std::max(int(t.n_u) + nd, 1)));
    k_merge_lists<<<nblk(nleaf + 1, 128), 128, 0, st>>>(nleaf, t.u_off, t.u_idx, t.d_off, t.d_idx, t.m_off,
                                                         t.m_idx);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    // -- statistics
    unsigned long long *d_pairs;
    int *d_max;
    RPY_TRY(dev_alloc(scratch, (void **)&d_pairs, 2 * sizeof(unsigned long long)));
    RPY_TRY(dev_alloc(scratch, (void **)&d_max, 2 * sizeof(int)));
    RPY_CHECK(cudaMemsetAsync(d_pairs, 0, 2 * sizeof(unsigned long long), st));
    RPY_CHECK(cudaMemsetAsync(d_max, 0, 2 * sizeof(int), st));
    k_leaf_stats<<<nblk(nleaf, 256), 256, 0, st>>>(nleaf, t.leaves, t.b_begin, t.b_end, t.u_off, t.u_idx, t.d_off,
                                                   t.d_idx, t.params.leaf_cap, d_pairs, d_max, d_max + 1);
    RPY_LAUNCHED(1);
    unsigned long long pairs[2] = {0, 0};
    int mx[2] = {0, 0};
    RPY_CHECK(cudaMemcpyAsync(pairs, d_pairs, sizeof(pairs), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaMemcpyAsync(mx, d_max, sizeof(mx), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaMemcpyAsync(&status, t.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    t.u_pairs = int64_t(pairs[0]);
    t.d_pairs = int64_t(pairs[1]);
    t.max_leaf_count = mx[0];
    t.leaves_over_cap = mx[1];
    // -- near-field work items in decreasing cost order
    {
        int *icnt, *ioff;
        RPY_TRY(dev_alloc(scratch, (void **)&icnt, sizeof(int) * (nleaf + 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&ioff, sizeof(int) * (nleaf + 1)));
        k_item_count<<<nblk(nleaf + 1, 256), 256, 0, st>>>(nleaf, t.leaves, t.b_begin, t.b_end, icnt);
        RPY_LAUNCHED(1);
        int ni = 0;
        if (scan_tmp_bytes(nleaf + 1) > sbytes) return RPY_ERR_INTERNAL;
        RPY_TRY(exclusive_scan_i32(icnt, ioff, nleaf + 1, &ni, stmp, sbytes, st));
        t.n_items = ni;
        int2 *items;
        uint64_t *ku, *kd, *km, *kt;
        uint32_t *vu, *vd, *vm, *vt;
        int *icounts;
        const int itiles = nblk(std::max(ni, 1), kSortTile);
        RPY_TRY(dev_alloc(scratch, (void **)&items, sizeof(int2) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&ku, sizeof(uint64_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&kd, sizeof(uint64_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&km, sizeof(uint64_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&kt, sizeof(uint64_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&vu, sizeof(uint32_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&vd, sizeof(uint32_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&vm, sizeof(uint32_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&vt, sizeof(uint32_t) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(scratch, (void **)&icounts, sizeof(int) * 256 * size_t(itiles)));
        if (scan_tmp_bytes(256 * itiles) > sbytes) return RPY_ERR_INTERNAL;
        RPY_TRY(dev_alloc(t, (void **)&t.u_items, sizeof(int2) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(t, (void **)&t.d_items, sizeof(int2) * std::max(ni, 1)));
        RPY_TRY(dev_alloc(t, (void **)&t.m_items, sizeof(int2) * std::max(ni, 1)));
        if (ni > 0) {
            k_item_fill<<<nblk(nleaf, 256), 256, 0, st>>>(nleaf, t.leaves, t.b_begin, t.b_end, t.u_off, t.u_idx,
                                                          t.d_off, t.d_idx, ioff, items, ku, vu, kd, vd, km, vm);
            RPY_LAUNCHED(1);
            RPY_TRY(radix_sort(ku, vu, kt, vt, ni, 8, icounts, stmp, sbytes, st));
            RPY_TRY(radix_sort(kd, vd, kt, vt, ni, 8, icounts, stmp, sbytes, st));
            RPY_TRY(radix_sort(km, vm, kt, vt, ni, 8, icounts, stmp, sbytes, st));
            k_item_order<<<nblk(ni, 256), 256, 0, st>>>(ni, items, vu, vd, vm, t.u_items, t.d_items, t.m_items);
            RPY_LAUNCHED(1);
            RPY_CHECK(cudaGetLastError());
        }
    }
    tree_release(scratch);
    if (status & DEVERR_STACK) return RPY_ERR_INTERNAL;
    return RPY_OK;
}

// ---------------------------------------------------------------- allocation-free bounding cube
//
// A variant of the bounding-cube reduction (k_bbox_partial / k_bbox_final)
// for callers that must not allocate device memory (for example code that
// runs while a caller-owned memory pool is locked, or inside a real-time
// step loop that forbids cudaMalloc).  Its per-chunk partials live in a
// fixed file-scope device array instead of a cudaMalloc'd buffer.

constexpr int kNoAllocMaxChunks = 4096;                                   // chunks of kChunk beads
constexpr int64_t kNoAllocMaxBeads = int64_t(kNoAllocMaxChunks) * kChunk;  // 33,554,432 beads
// per chunk: lo xyz, hi xyz, non-finite flag
static __device__ __align__(256) double g_cube_scratch[kNoAllocMaxChunks * 7];

static std::mutex g_cube_mu;
static void *g_cube_ptr[256] = {};

__global__ void k_bbox_partial_fixed(const double *pos, int64_t n, double *part) {
    __shared__ double red[7][256];
    int64_t c0 = int64_t(blockIdx.x) * kChunk;
    int64_t c1 = c0 + kChunk < n ? c0 + kChunk : n;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double bad = 0.0;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double v = pos[3 * i + a];
            if (!isfinite(v)) bad = 1.0;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = lo[a];
        red[3 + a][threadIdx.x] = hi[a];
    }
    red[6][threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + s]);
                red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + s]);
            }
            red[6][threadIdx.x] = fmax(red[6][threadIdx.x], red[6][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) part[7 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// One block: reduce nch partials, then the cube exactly as k_bbox_final.
__global__ void k_bbox_final_fixed(const double *part, int nch, double *cube) {
    __shared__ double red[7][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double bad = 0.0;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], part[7 * c + a]);
            hi[a] = fmax(hi[a], part[7 * c + 3 + a]);
        }
        bad = fmax(bad, part[7 * c + 6]);
    }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = lo[a];
        red[3 + a][threadIdx.x] = hi[a];
    }
    red[6][threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + s]);
                red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + s]);
            }
            red[6][threadIdx.x] = fmax(red[6][threadIdx.x], red[6][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double side = 0.0;
        for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(red[3 + a][0], red[a][0]));
        for (int a = 0; a < 3; ++a) cube[a] = __dmul_rn(0.5, __dadd_rn(red[a][0], red[3 + a][0]));
        cube[3] = red[6][0] != 0.0 ? NAN : side;
    }
}

int bounding_cube_noalloc(const double *pos_dev, int64_t n, double *cube_dev, cudaStream_t st) {
    if (n > kNoAllocMaxBeads) {
        set_last_error("rpy_bounding_cube_noalloc: n exceeds the fixed scratch limit of 33554432 beads");
        return RPY_ERR_INVALID;
    }
    int dev = 0;
    RPY_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return RPY_ERR_INVALID;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_cube_mu);
        if (!g_cube_ptr[dev]) {
            // host code only knows a stand-in for the array: ask the runtime for
            // its address on this device (the current one) once
            void *ptr = nullptr;
            RPY_CHECK(cudaGetSymbolAddress(&ptr, g_cube_scratch));
            g_cube_ptr[dev] = ptr;
        }
        scratch = g_cube_ptr[dev];
    }
    int nch = int((n + kChunk - 1) / kChunk);
    k_bbox_partial_fixed<<<nch, 256, 0, st>>>(pos_dev, n, static_cast<double *>(scratch));
    RPY_LAUNCHED(1);
    k_bbox_final_fixed<<<1, 256, 0, st>>>(static_cast<const double *>(scratch), nch, cube_dev);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    return RPY_OK;
}

int tree_build_vlists(Tree &t, cudaStream_t st) {
    if (t.v_off) return RPY_OK;
    int nbx = t.nbox;
    Tree scratch;
    scratch.owner = &t;
    int *vcnt;
    void *stmp;
    size_t sbytes = scan_tmp_bytes(nbx + 1);
    RPY_TRY(dev_alloc(scratch, (void **)&vcnt, sizeof(int) * (nbx + 1)));
    RPY_TRY(dev_alloc(scratch, &stmp, sbytes));
    RPY_CHECK(cudaMemsetAsync(vcnt, 0, sizeof(int) * (nbx + 1), st));
    k_vlists<false><<<nblk(nbx, 128), 128, 0, st>>>(0, nbx, t.b_level, t.b_parent, t.b_child, t.b_coll, t.b_cell,
                                                    t.b_leaf, vcnt, nullptr, nullptr);
    RPY_LAUNCHED(1);
    RPY_TRY(dev_alloc(t, (void **)&t.v_off, sizeof(int) * (nbx + 1)));
    int nv = 0;
    RPY_TRY(exclusive_scan_i32(vcnt, t.v_off, nbx + 1, &nv, stmp, sbytes, st));
    t.n_v = nv;
    RPY_TRY(dev_alloc(t, (void **)&t.v_idx, sizeof(int) * std::max(nv, 1)));
    k_vlists<true><<<nblk(nbx, 128), 128, 0, st>>>(0, nbx, t.b_level, t.b_parent, t.b_child, t.b_coll, t.b_cell,
                                                   t.b_leaf, nullptr, t.v_off, t.v_idx);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_CHECK(cudaStreamSynchronize(st));
    tree_release(scratch);
    return RPY_OK;
}

}  // namespace rpy
