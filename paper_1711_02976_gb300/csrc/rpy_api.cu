// C ABI of librpyfmm (see include/rpyfmm.h for the contract of every entry point).
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <atomic>
#include <tuple>

#include "rpy_internal.h"

struct rpy_tree_s {
    rpy::Tree t;
    unsigned magic = 0x52505954u;
};

namespace rpy {

static constexpr double kPiA = 3.14159265358979323846;

// ---------------------------------------------------------------- kernels used here

// Forces into sorted SoA; the FP32 form also keeps a single-precision copy.
__global__ void k_gather_f(const double *f, const int *perm, int64_t n, double *fs, float *f32) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    double fx = f[3 * j], fy = f[3 * j + 1], fz = f[3 * j + 2];
    fs[i] = fx;
    fs[n + i] = fy;
    fs[2 * n + i] = fz;
    if (f32) {
        f32[i] = float(fx);
        f32[n + i] = float(fy);
        f32[2 * n + i] = float(fz);
    }
}

__global__ void k_pair_const(int nsys, const double *a_, const double *s_, const double *cube, PairConst *pc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsys) return;
    const double a = a_[k], s = s_[k];
    PairConst c;
    c.a = a;
    c.co = s / (6.0 * kPiA * a);
    c.cf = s / (8.0 * kPiA);
    c.k23 = 2.0 * a * a / 3.0;
    c.nk2 = -2.0 * a * a;
    c.a2x4 = 4.0 * a * a;
    c.C1 = s / (8.0 * kPiA);
    c.C2 = s * a * a / (12.0 * kPiA);
    c.icube = 1.0 / cube[4 * k + 3];
    const double co_cf = c.co / c.cf;
    c.f_a2x4 = float(c.a2x4);
    c.f_tiny2 = fmaxf(float(1e-6 * a * a), 1e-36f);   // a normal FP32 number
    c.f_k23 = float(c.k23);
    c.f_nk2 = float(c.nk2);
    c.f_co_cf = float(co_cf);
    c.f_nco_c9 = float(-co_cf * 9.0 / (32.0 * a));
    c.f_co_c3 = float(co_cf * 3.0 / (32.0 * a));
    c.f_pad = 0.f;
    pc[k] = c;
}

__global__ void k_gather_q4(const double *q, const int *perm, int64_t n, double *qs) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int k = 0; k < 4; ++k) qs[4 * i + k] = q[4 * j + k];
}

__global__ void k_combine(const int *perm, int64_t n, const double *un, const double *uf, const double *ud, int parts,
                          double *u) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        if (parts & RPY_PART_NEAR) v += un[3 * i + a];
        if (parts & RPY_PART_FAR) v += uf[3 * i + a] + (ud ? ud[3 * i + a] : 0.0);
        u[3 * j + a] = v;
    }
}

__global__ void k_unperm_lap(const int *perm, int64_t n, const double *src, double *dst) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int c = 0; c < 52; ++c) dst[52 * j + c] = src[52 * i + c];
}

static inline int nb256(int64_t n) { return int((n + 255) / 256); }

// FMA throughput probe: 8 independent dependency chains per thread.
template <typename T>
__global__ void k_fma_probe(T *out, int iters, T a, T b) {
    T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// ---------------------------------------------------------------- instrumentation

static std::atomic<int64_t> g_launches{0};
void note_launches(int n) { g_launches += n; }

void prof_mark(Tree &t, int k, cudaStream_t st) {
    if (!t.prof || k < 0 || k > RPY_NUM_STAGES || t.n_marks >= Tree::kMaxMarks) return;
    const int i = t.n_marks++;
    if (!t.ev[i]) cudaEventCreate(&t.ev[i]);
    cudaEventRecord(t.ev[i], st);
    t.ev_stage[i] = k;
}

// ---------------------------------------------------------------- table cache

struct DevTableSet {
    void *mem = nullptr;
    DevTables<double> d64{};
    DevTables<float> d32{};
};

static std::mutex g_mu;
static std::map<std::tuple<int, int, int>, OpTables *> g_host_tabs;      // (p, quadrature rule, 0)
static std::map<std::tuple<int, int, int>, DevTableSet *> g_dev_tabs;    // (device, p, quadrature rule)

static int host_tables(int p, int digits, OpTables **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(p, digits, 0);
    auto it = g_host_tabs.find(key);
    if (it != g_host_tabs.end()) {
        *out = it->second;
        return RPY_OK;
    }
    OpTables *t = new (std::nothrow) OpTables();
    if (!t) return RPY_ERR_INTERNAL;
    int s = build_tables(p, digits, *t);
    if (s != RPY_OK) {
        delete t;
        return s;
    }
    g_host_tabs[key] = t;
    *out = t;
    return RPY_OK;
}

// Upload one table set in both precisions into a single device block.
template <typename T>
static void pack_tables(const OpTables &h, std::vector<char> &blob, std::vector<size_t> &offs) {
    auto put = [&](const void *src, size_t bytes) {
        size_t o = (blob.size() + 255) / 256 * 256;
        blob.resize(o + bytes);
        if (bytes) std::memcpy(blob.data() + o, src, bytes);
        offs.push_back(o);
    };
    auto putT = [&](const std::vector<double> &v) {
        std::vector<T> c(v.begin(), v.end());
        put(c.data(), sizeof(T) * c.size());
    };
    auto putI = [&](const std::vector<int> &v) { put(v.data(), sizeof(int) * v.size()); };
    putT(h.m2m_t);    // 0
    putT(h.l2l_t);    // 1
    putT(h.rot_fwd);  // 2
    putT(h.rot_bwd);  // 3
    putI(h.rot_off);  // 4
    putT(h.rec_a);    // 5
    putT(h.rec_b);    // 6
    putT(h.rec_c);    // 7
    putT(h.rec_cm);   // 8
    putT(h.roots);    // 9
    putT(h.m2x_c);    // 10
    putT(h.x2l_c);    // 11
    putI(h.e_k);      // 12
    putI(h.k_start);  // 13
    putT(h.e_cos);    // 14
    putT(h.e_sin);    // 15
    putT(h.e_wm);     // 16
    putT(h.shift);    // 17
    putI(h.grp_off);  // 18
    putI(h.grp_n);    // 19
    putI(h.grp_mask); // 20
    putI(h.slot_list);// 21
    putI(h.child_shift); // 22
    putT(h.lad);      // 23
    putT(h.orot_fwd); // 24
    putT(h.orot_bwd); // 25
    putT(h.zm2m);     // 26
    putT(h.zl2l);     // 27
    putT(h.frot_fwd); // 28
    putT(h.frot_bwd); // 29
    putT(h.forot_fwd);// 30
    putT(h.forot_bwd);// 31
    putI(h.frot_off); // 32
    putI(h.u_k);      // 33
    putI(h.u_start);  // 34
    putT(h.shz);      // 35
    putT(h.shx);      // 36
    putT(h.shy);      // 37
    {                 // 38: shift rows padded to an even length
        const int S = h.S, Sp = (S + 1) & ~1;
        std::vector<double> v(size_t(216) * Sp * 2, 0.0);
        for (int o = 0; o < 216; ++o)
            for (int e = 0; e < 2 * S; ++e) v[size_t(o) * Sp * 2 + e] = h.shift[size_t(o) * S * 2 + e];
        putT(v);
    }
}

template <typename T>
static DevTables<T> bind_tables(const OpTables &h, char *base, const std::vector<size_t> &o) {
    DevTables<T> d{};
    d.p = h.p;
    d.nc = h.nc;
    d.s = h.s;
    d.S = h.S;
    d.rot_len = h.rot_off.back();
    d.m2m_t = reinterpret_cast<const T *>(base + o[0]);
    d.l2l_t = reinterpret_cast<const T *>(base + o[1]);
    d.rot_fwd = reinterpret_cast<const T *>(base + o[2]);
    d.rot_bwd = reinterpret_cast<const T *>(base + o[3]);
    d.rot_off = reinterpret_cast<const int *>(base + o[4]);
    d.rec_a = reinterpret_cast<const T *>(base + o[5]);
    d.rec_b = reinterpret_cast<const T *>(base + o[6]);
    d.rec_c = reinterpret_cast<const T *>(base + o[7]);
    d.rec_cm = reinterpret_cast<const T *>(base + o[8]);
    d.roots = reinterpret_cast<const cpx<T> *>(base + o[9]);
    d.m2x_c = reinterpret_cast<const T *>(base + o[10]);
    d.x2l_c = reinterpret_cast<const T *>(base + o[11]);
    d.e_k = reinterpret_cast<const int *>(base + o[12]);
    d.k_start = reinterpret_cast<const int *>(base + o[13]);
    d.e_cos = reinterpret_cast<const T *>(base + o[14]);
    d.e_sin = reinterpret_cast<const T *>(base + o[15]);
    d.e_wm = reinterpret_cast<const T *>(base + o[16]);
    d.shift = reinterpret_cast<const cpx<T> *>(base + o[17]);
    d.grp_off = reinterpret_cast<const int *>(base + o[18]);
    d.grp_n = reinterpret_cast<const int *>(base + o[19]);
    d.grp_mask = reinterpret_cast<const int *>(base + o[20]);
    d.slot_list = reinterpret_cast<const int *>(base + o[21]);
    d.child_shift = reinterpret_cast<const int *>(base + o[22]);
    d.lad = reinterpret_cast<const T *>(base + o[23]);
    d.orot_fwd = reinterpret_cast<const T *>(base + o[24]);
    d.orot_bwd = reinterpret_cast<const T *>(base + o[25]);
    d.zm2m = reinterpret_cast<const T *>(base + o[26]);
    d.zl2l = reinterpret_cast<const T *>(base + o[27]);
    d.frot_fwd = reinterpret_cast<const T *>(base + o[28]);
    d.frot_bwd = reinterpret_cast<const T *>(base + o[29]);
    d.forot_fwd = reinterpret_cast<const T *>(base + o[30]);
    d.forot_bwd = reinterpret_cast<const T *>(base + o[31]);
    d.frot_off = reinterpret_cast<const int *>(base + o[32]);
    d.frot_len = h.frot_off.back();
    d.u_k = reinterpret_cast<const int *>(base + o[33]);
    d.u_start = reinterpret_cast<const int *>(base + o[34]);
    d.NU = int(h.u_k.size());
    d.shz = reinterpret_cast<const T *>(base + o[35]);
    d.shx = reinterpret_cast<const cpx<T> *>(base + o[36]);
    d.shy = reinterpret_cast<const cpx<T> *>(base + o[37]);
    d.shiftp = reinterpret_cast<const cpx<T> *>(base + o[38]);
    d.Sp = (h.S + 1) & ~1;
    return d;
}

static int device_tables(int dev, int p, int digits, DevTableSet **out) {
    OpTables *h = nullptr;
    RPY_TRY(host_tables(p, digits, &h));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(dev, p, digits);
    auto it = g_dev_tabs.find(key);
    if (it != g_dev_tabs.end()) {
        *out = it->second;
        return RPY_OK;
    }
    std::vector<char> b64, b32;
    std::vector<size_t> o64, o32;
    pack_tables<double>(*h, b64, o64);
    pack_tables<float>(*h, b32, o32);
    size_t off32 = (b64.size() + 255) / 256 * 256;
    void *mem = nullptr;
    RPY_CHECK(cudaMalloc(&mem, off32 + b32.size()));
    cudaError_t e1 = cudaMemcpy(mem, b64.data(), b64.size(), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(static_cast<char *>(mem) + off32, b32.data(), b32.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFree(mem);
        return check_cuda("table upload", e1 != cudaSuccess ? e1 : e2);
    }
    DevTableSet *s = new DevTableSet();
    s->mem = mem;
    s->d64 = bind_tables<double>(*h, static_cast<char *>(mem), o64);
    s->d32 = bind_tables<float>(*h, static_cast<char *>(mem) + off32, o32);
    g_dev_tabs[key] = s;
    *out = s;
    return RPY_OK;
}

// ---------------------------------------------------------------- helpers


static int have_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return RPY_ERR_NODEVICE;
    }
    return RPY_OK;
}

// Completion tracking: an event owned by the tree, recorded after each call.
static void mark_done(Tree &t, cudaStream_t st) {
    if (!t.done) cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming);
    cudaEventRecord(t.done, st);
    t.last_stream = st;
}

static cudaError_t wait_done(Tree &t) { return t.done ? cudaEventSynchronize(t.done) : cudaSuccess; }

static bool valid(rpy_tree t) { return t && t->magic == 0x52505954u; }

Tree *tree_of(rpy_tree h) { return valid(h) ? &h->t : nullptr; }

static int alloc_tree_arrays(Tree &t, cudaStream_t st) {
    int64_t n = t.n;
    RPY_TRY(dev_alloc(t, (void **)&t.sys_off, sizeof(int64_t) * (t.nsys + 1)));
    RPY_TRY(dev_alloc(t, (void **)&t.sys_a, sizeof(double) * t.nsys));
    RPY_TRY(dev_alloc(t, (void **)&t.sys_s, sizeof(double) * t.nsys));
    RPY_TRY(dev_alloc(t, (void **)&t.sys_pc, sizeof(PairConst) * t.nsys));
    RPY_TRY(dev_alloc(t, (void **)&t.sys_cube, sizeof(double) * 4 * t.nsys));
    RPY_TRY(dev_alloc(t, (void **)&t.perm, sizeof(int) * n));
    RPY_TRY(dev_alloc(t, (void **)&t.keys, sizeof(uint64_t) * n));
    RPY_TRY(dev_alloc(t, (void **)&t.pos, sizeof(double) * 3 * n));
    RPY_TRY(dev_alloc(t, (void **)&t.bead_sys, sizeof(int) * n));
    RPY_TRY(dev_alloc(t, (void **)&t.dev_status, sizeof(unsigned)));
    RPY_CHECK(cudaMemcpyAsync(t.sys_off, t.sys_off_h.data(), sizeof(int64_t) * (t.nsys + 1), cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(t.sys_a, t.a_h.data(), sizeof(double) * t.nsys, cudaMemcpyHostToDevice, st));
    t.sys_s_h.assign(t.nsys, NAN);
    return RPY_OK;
}

int tree_alloc_workspace(Tree &t, cudaStream_t st) {
    const OpTables &h = *t.tabs;
    size_t es = t.params.precision == RPY_FP32 ? sizeof(cpx<float>) : sizeof(cpx<double>);
    size_t nb = size_t(t.nbox);
    if (t.params.flags & RPY_FLAG_CARTESIAN) {
        // real coefficients: multipoles and locals of four sets, three velocity polynomials per leaf
        const size_t rs = es / 2, N = size_t(cart_terms(t.p));
        RPY_TRY(tree_build_vlists(t, st));
        RPY_TRY(dev_alloc(t, &t.M, rs * nb * kSets * N));
        RPY_TRY(dev_alloc(t, &t.L, rs * nb * kSets * N));
        RPY_TRY(dev_alloc(t, &t.EVg, rs * size_t(t.nleaf) * 3 * N));
        RPY_TRY(dev_alloc(t, (void **)&t.fs, sizeof(double) * 3 * t.n));
        if (t.params.precision == RPY_FP32) {
            RPY_TRY(dev_alloc(t, (void **)&t.p32, sizeof(float) * 6 * t.n));
            RPY_TRY(dev_alloc(t, (void **)&t.f32, sizeof(float) * 3 * t.n));
        }
        RPY_TRY(dev_alloc(t, (void **)&t.u_near, sizeof(double) * 3 * t.n));
        RPY_TRY(dev_alloc(t, (void **)&t.u_far, sizeof(double) * 3 * t.n));
        RPY_TRY(dev_alloc(t, (void **)&t.u_dir, sizeof(double) * 3 * t.n));
        return RPY_OK;
    }
    RPY_TRY(dev_alloc(t, &t.M, es * nb * kSets * h.nc));
    RPY_TRY(dev_alloc(t, &t.L, es * nb * kSets * h.nc));
    t.x_frames = (t.params.flags & RPY_FLAG_FRAME_PASSES) ? 1 : plane_wave_frames(double(nb), double(es), h.S);
    RPY_TRY(dev_alloc(t, &t.Xo, es * nb * 2 * t.x_frames * kSets * h.S));
    RPY_TRY(dev_alloc(t, &t.Xi, es * nb * 2 * t.x_frames * kSets * h.S));
    RPY_TRY(dev_alloc(t, &t.EVg, es * size_t(t.nleaf) * 18 * h.nc));
    if (t.params.precision != RPY_FP32 || h.p >= 12) {   // rotation-based M2M (see run_far_t)
        size_t wide = 0;   // the widest parent level of the M2M pass (levels 2 .. nlevels - 2)
        for (int l = 2; l <= t.nlevels - 2; ++l)
            wide = std::max(wide, size_t(t.level_off[l + 1] - t.level_off[l]));
        if (wide > 0) RPY_TRY(dev_alloc(t, &t.m2m_scratch, es * wide * 8 * kSets * h.nc));
    }
    RPY_TRY(dev_alloc(t, (void **)&t.fs, sizeof(double) * 3 * t.n));
    if (t.params.precision == RPY_FP32) {
        RPY_TRY(dev_alloc(t, (void **)&t.p32, sizeof(float) * 6 * t.n));
        RPY_TRY(dev_alloc(t, (void **)&t.f32, sizeof(float) * 3 * t.n));
    }
    RPY_TRY(dev_alloc(t, (void **)&t.u_near, sizeof(double) * 3 * t.n));
    RPY_TRY(dev_alloc(t, (void **)&t.u_far, sizeof(double) * 3 * t.n));
    RPY_TRY(dev_alloc(t, (void **)&t.u_dir, sizeof(double) * 3 * t.n));
    return RPY_OK;
}

static int do_build(Tree &t, const double *pos_dev, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    t.built = false;
    RPY_TRY(alloc_tree_arrays(t, st));
    RPY_TRY(tree_build(t, pos_dev, st));
    OpTables *h = nullptr;
    RPY_TRY(host_tables(t.p, t.params.quad, &h));
    t.tabs = h;   // the host description (sizes used by workspace / stats), cached for the process
    DevTableSet *ds = nullptr;
    RPY_TRY(device_tables(t.device, t.p, t.params.quad, &ds));
    t.dt64 = ds->d64;
    t.dt32 = ds->d32;
    RPY_TRY(tree_alloc_workspace(t, st));
    if (t.params.precision == RPY_FP32) RPY_TRY(split_positions_f32(t, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    mark_done(t, st);
    t.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    t.built = true;
    return RPY_OK;
}

static int upload_s(Tree &t, const double *s_host, cudaStream_t st) {
    bool same = true;
    for (int k = 0; k < t.nsys; ++k)
        if (!(t.sys_s_h[k] == s_host[k])) same = false;
    if (same) return RPY_OK;
    // the copy is ordered on st before every kernel that reads it
    RPY_CHECK(cudaMemcpyAsync(t.sys_s, s_host, sizeof(double) * t.nsys, cudaMemcpyHostToDevice, st));
    k_pair_const<<<(t.nsys + 127) / 128, 128, 0, st>>>(t.nsys, t.sys_a, t.sys_s, t.sys_cube, t.sys_pc);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    RPY_CHECK(cudaStreamSynchronize(st));
    t.sys_s_h.assign(s_host, s_host + t.nsys);
    return RPY_OK;
}

// Body of the matvec on stream st: near field, direct substitutes, far field.
// With `side` (the captured graph) the two pair passes run on side_stream
// beside the far-field chain and are joined back into st at the end; the
// stage-timing path keeps them in sequence.
static int matvec_body(Tree &t, const SysConst &sc, int parts, cudaStream_t st, bool side = false) {
    cudaStream_t sp = st;
    if (side) {
        RPY_CHECK(cudaEventRecord(t.fork_ev, st));
        RPY_CHECK(cudaStreamWaitEvent(t.side_stream, t.fork_ev, 0));
        sp = t.side_stream;
    }
    prof_mark(t, RPY_STAGE_P2P, st);
    if (parts == RPY_PART_ALL) {
        // one pass over each leaf's U list and direct substitutes (u_dir stays zero)
        RPY_TRY(run_p2p(t, t.fs, t.u_near, sc, sp, kListM));
    } else {
        if (parts & RPY_PART_NEAR) RPY_TRY(run_p2p(t, t.fs, t.u_near, sc, sp, kListU));
        if (parts & RPY_PART_FAR) RPY_TRY(run_p2p(t, t.fs, t.u_dir, sc, sp, kListD));
    }
    prof_mark(t, RPY_STAGE_P2M, st);
    if (parts & RPY_PART_FAR) {
        if (t.params.flags & RPY_FLAG_CARTESIAN) {
            if (t.params.precision == RPY_FP32) RPY_TRY(run_cart_t<float>(t, t.fs, t.u_far, sc, st));
            else RPY_TRY(run_cart_t<double>(t, t.fs, t.u_far, sc, st));
        } else if (t.params.precision == RPY_FP32) {
            RPY_TRY(run_far_t<float>(t, t.dt32, t.fs, nullptr, t.u_far, nullptr, sc, st));
        } else {
            RPY_TRY(run_far_t<double>(t, t.dt64, t.fs, nullptr, t.u_far, nullptr, sc, st));
        }
    }
    if (side) {
        RPY_CHECK(cudaEventRecord(t.join_ev, t.side_stream));
        RPY_CHECK(cudaStreamWaitEvent(st, t.join_ev, 0));
    }
    return RPY_OK;
}

static void drop_graph(Tree &t) {
    if (t.gexec) cudaGraphExecDestroy(t.gexec);
    t.gexec = nullptr;
}

// Capture the matvec body once on the tree's own stream (capture on the legacy
// stream is not allowed) and keep the instantiated graph.
static int capture_graph(Tree &t, const SysConst &sc) {
    if (!t.cap_stream) RPY_CHECK(cudaStreamCreateWithFlags(&t.cap_stream, cudaStreamNonBlocking));
    if (!t.side_stream) RPY_CHECK(cudaStreamCreateWithFlags(&t.side_stream, cudaStreamNonBlocking));
    if (!t.fork_ev) RPY_CHECK(cudaEventCreateWithFlags(&t.fork_ev, cudaEventDisableTiming));
    if (!t.join_ev) RPY_CHECK(cudaEventCreateWithFlags(&t.join_ev, cudaEventDisableTiming));
    RPY_CHECK(cudaStreamBeginCapture(t.cap_stream, cudaStreamCaptureModeThreadLocal));
    int s = matvec_body(t, sc, RPY_PART_ALL, t.cap_stream, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(t.cap_stream, &g);
    if (s != RPY_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return check_cuda("cudaStreamEndCapture", e);
    e = cudaGraphInstantiate(&t.gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        t.gexec = nullptr;
        return check_cuda("cudaGraphInstantiate", e);
    }
    return RPY_OK;
}

int run_matvec(Tree &t, const double *f_dev, const double *s_host, double *u_dev, int parts, cudaStream_t st) {
    if (!t.built) return RPY_ERR_STATE;
    RPY_TRY(upload_s(t, s_host, st));
    SysConst sc{t.sys_cube, t.sys_a, t.sys_s, t.sys_pc};
    t.n_marks = 0;
    prof_mark(t, RPY_STAGE_GATHER, st);
    k_gather_f<<<nb256(t.n), 256, 0, st>>>(f_dev, t.perm, t.n, t.fs, t.f32);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    bool graph = parts == RPY_PART_ALL && !t.prof && !(t.params.flags & RPY_FLAG_NO_GRAPH) && t.matvecs >= 1;
    if (graph && !t.gexec) RPY_TRY(capture_graph(t, sc));
    if (graph) {
        RPY_CHECK(cudaGraphLaunch(t.gexec, st));
        RPY_LAUNCHED(1);
    } else {
        RPY_TRY(matvec_body(t, sc, parts, st));
    }
    prof_mark(t, RPY_STAGE_COMBINE, st);
    // the full matvec summed the direct substitutes into u_near
    k_combine<<<nb256(t.n), 256, 0, st>>>(t.perm, t.n, t.u_near, t.u_far, parts == RPY_PART_ALL ? nullptr : t.u_dir,
                                          parts, u_dev);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    prof_mark(t, RPY_NUM_STAGES, st);
    mark_done(t, st);
    t.matvecs++;
    return RPY_OK;
}

int run_laplace_far(Tree &t, const double *q_dev, double *out_dev, cudaStream_t st) {
    if (!t.built || (t.params.flags & RPY_FLAG_CARTESIAN)) return RPY_ERR_STATE;
    if (!std::isfinite(t.sys_s_h[0])) {   // per-system constants (their geometric part) for a tree never applied
        std::vector<double> one(t.nsys, 1.0);
        RPY_TRY(upload_s(t, one.data(), st));
    }
    if (!t.lap_q) {
        RPY_TRY(dev_alloc(t, (void **)&t.lap_q, sizeof(double) * 4 * t.n));
    }
    double *lap_out = nullptr;
    Tree scratch;
    RPY_TRY(dev_alloc(scratch, (void **)&lap_out, sizeof(double) * 52 * t.n));
    SysConst sc{t.sys_cube, t.sys_a, t.sys_s, t.sys_pc};
    k_gather_q4<<<nb256(t.n), 256, 0, st>>>(q_dev, t.perm, t.n, t.lap_q);
    RPY_LAUNCHED(1);
    int s;
    if (t.params.precision == RPY_FP32)
        s = run_far_t<float>(t, t.dt32, nullptr, t.lap_q, nullptr, lap_out, sc, st);
    else
        s = run_far_t<double>(t, t.dt64, nullptr, t.lap_q, nullptr, lap_out, sc, st);
    if (s == RPY_OK) {
        k_unperm_lap<<<nb256(t.n), 256, 0, st>>>(t.perm, t.n, lap_out, out_dev);
        RPY_LAUNCHED(1);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = check_cuda("laplace far", e);
    }
    tree_release(scratch);
    mark_done(t, st);
    return s;
}

static int check_params(const rpy_build_params &p) {
    if (p.digits != 3 && p.digits != 6 && p.digits != 9) return RPY_ERR_DIGITS;
    if (p.precision != RPY_FP64 && p.precision != RPY_FP32) return RPY_ERR_INVALID;
    if (p.digits == 9 && p.precision != RPY_FP64) return RPY_ERR_DIGITS;   // beyond FP32 arithmetic
    if (p.leaf_cap < 0 || p.order_p < 0 || p.max_level < 0 || p.max_level > kMaxLevel ||
        (p.flags & ~(RPY_FLAG_NO_GRAPH | RPY_FLAG_FRAME_PASSES | RPY_FLAG_EVAL_PER_POTENTIAL |
                     RPY_FLAG_BOX_ORIGIN | RPY_FLAG_CUBE_ORIGIN | RPY_FLAG_CARTESIAN)) != 0 ||
        ((p.flags & RPY_FLAG_BOX_ORIGIN) && (p.flags & RPY_FLAG_CUBE_ORIGIN)))
        return RPY_ERR_INVALID;
    if (p.order_p != 0 && (p.order_p < 2 || p.order_p > kMaxP)) return RPY_ERR_INVALID;
    if (p.flags & RPY_FLAG_CARTESIAN) {
        if (p.digits != 3) return RPY_ERR_DIGITS;
        if (p.order_p > kCartMaxP) return RPY_ERR_INVALID;
    }
    if (p.direct_w < -1 || p.direct_x < -1) return RPY_ERR_INVALID;
    if (p.quad != 0 && (p.quad < 3 || p.quad > 6) && p.quad != 9) return RPY_ERR_INVALID;
    return RPY_OK;
}

}  // namespace rpy

using namespace rpy;

extern "C" {

int rpy_version(void) { return 100; }

const char *rpy_strerror(int status) {
    switch (status) {
        case RPY_OK: return "success";
        case RPY_ERR_INVALID: return "invalid argument";
        case RPY_ERR_DIGITS: return "digits must be 3, 6 or 9";
        case RPY_ERR_OOM: return "device memory allocation failed";
        case RPY_ERR_CUDA: return "CUDA error";
        case RPY_ERR_TIMEOUT: return "device wait timed out";
        case RPY_ERR_NONFINITE: return "non-finite position";
        case RPY_ERR_STATE: return "handle in wrong state";
        case RPY_ERR_NODEVICE: return "no CUDA device";
        case RPY_ERR_INTERNAL: return "internal capacity exceeded";
        default: return "unknown status";
    }
}

const char *rpy_last_cuda_error(void) { return last_cuda_error_text(); }

int rpy_forest_build(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                     const rpy_build_params *params, void *stream, rpy_tree *out) {
    if (!out) return RPY_ERR_INVALID;
    *out = nullptr;
    if (!pos_dev || !sys_offsets || !a_host || !params || nsys < 1) return RPY_ERR_INVALID;
    RPY_TRY(check_params(*params));
    if (sys_offsets[0] != 0) return RPY_ERR_INVALID;
    for (int k = 0; k < nsys; ++k) {
        if (sys_offsets[k + 1] <= sys_offsets[k]) return RPY_ERR_INVALID;
        if (!(a_host[k] > 0.0) || !std::isfinite(a_host[k])) return RPY_ERR_INVALID;
    }
    if (sys_offsets[nsys] > int64_t(0x7fffffff) / 2) return RPY_ERR_INVALID;
    RPY_TRY(have_device());
    rpy_tree h = new (std::nothrow) rpy_tree_s();
    if (!h) return RPY_ERR_INTERNAL;
    Tree &t = h->t;
    cudaGetDevice(&t.device);
    t.n = sys_offsets[nsys];
    t.nsys = nsys;
    t.params = *params;
    if (t.params.leaf_cap == 0) t.params.leaf_cap = default_leaf_cap(params->digits);
    if (t.params.max_level == 0) t.params.max_level = kMaxLevel;
    if (t.params.quad == 0) t.params.quad = params->digits;
    t.p = params->order_p ? params->order_p : default_order(params->digits);
    t.direct_w = params->direct_w < 0 ? 0 : (params->direct_w > 0 ? params->direct_w : int(1.8 * ncoef(t.p + 2)));
    t.direct_x = params->direct_x < 0 ? 0 : (params->direct_x > 0 ? params->direct_x : int(0.6 * ncoef(t.p)));
    if (params->flags & RPY_FLAG_CARTESIAN) {
        // polynomial far field: no multipole-to-target or source-to-local operators, so every
        // W- and X-list interaction is summed directly
        if (!params->order_p) t.p = kCartDefaultP;
        t.direct_w = t.direct_x = 0x7fffffff;
    }
    t.sys_off_h.assign(sys_offsets, sys_offsets + nsys + 1);
    t.a_h.assign(a_host, a_host + nsys);
    int s = do_build(t, pos_dev, static_cast<cudaStream_t>(stream));
    if (s != RPY_OK) {
        tree_release(t);
        delete h;
        return s;
    }
    *out = h;
    return RPY_OK;
}

int rpy_tree_build(const double *pos_dev, int64_t n, double a, int digits, int leaf_cap, int precision, void *stream,
                   rpy_tree *out) {
    if (!out) return RPY_ERR_INVALID;
    *out = nullptr;
    if (n < 1) return RPY_ERR_INVALID;
    rpy_build_params p{};
    p.digits = digits;
    p.precision = precision;
    p.leaf_cap = leaf_cap;
    int64_t off[2] = {0, n};
    return rpy_forest_build(pos_dev, off, 1, &a, &p, stream, out);
}

int rpy_tree_update_positions(rpy_tree h, const double *pos_dev, void *stream) {
    if (!valid(h) || !pos_dev) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    wait_done(t);
    drop_graph(t);
    // keep handle-level settings and the device blocks (as a cache), rebuild the structures
    tree_recycle(t);
    Tree fresh;
    fresh.device = t.device;
    fresh.n = t.n;
    fresh.nsys = t.nsys;
    fresh.params = t.params;
    fresh.p = t.p;
    fresh.direct_w = t.direct_w;
    fresh.direct_x = t.direct_x;
    fresh.prof = t.prof;
    for (int k = 0; k < Tree::kMaxMarks; ++k) fresh.ev[k] = t.ev[k];
    fresh.done = t.done;
    fresh.cap_stream = t.cap_stream;
    fresh.side_stream = t.side_stream;
    fresh.fork_ev = t.fork_ev;
    fresh.join_ev = t.join_ev;
    fresh.h2d_ev = t.h2d_ev;
    fresh.sys_off_h = t.sys_off_h;
    fresh.a_h = t.a_h;
    fresh.cache = std::move(t.cache);
    fresh.device_bytes = t.device_bytes;
    fresh.host_io = t.host_io;
    t = std::move(fresh);
    return do_build(t, pos_dev, static_cast<cudaStream_t>(stream));
}

int rpy_tree_matvec_host(rpy_tree h, const double *pos_host, const double *f_host, const double *s_host,
                         double *u_host, void *stream) {
    if (!valid(h) || !f_host || !u_host || !s_host) return RPY_ERR_INVALID;
    Tree &t = h->t;
    for (int k = 0; k < t.nsys; ++k)
        if (!std::isfinite(s_host[k])) return RPY_ERR_INVALID;
    DeviceGuard g(t.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n3 = 3 * size_t(t.n);
    if (!t.host_io) {
        cudaError_t e = cudaMalloc(&t.host_io, sizeof(double) * 3 * n3);
        if (e != cudaSuccess) {
            t.host_io = nullptr;
            return check_cuda("cudaMalloc (host-buffer matvec)", e);
        }
    }
    double *dp = t.host_io, *df = t.host_io + n3, *du = t.host_io + 2 * n3;
    if (pos_host) {
        // the forces' copy on the side stream, beside the rebuild (the previous call of this
        // entry synchronised st, so nothing still reads df); st waits for it before the matvec
        if (!t.side_stream) RPY_CHECK(cudaStreamCreateWithFlags(&t.side_stream, cudaStreamNonBlocking));
        if (!t.h2d_ev) RPY_CHECK(cudaEventCreateWithFlags(&t.h2d_ev, cudaEventDisableTiming));
        RPY_CHECK(cudaMemcpyAsync(dp, pos_host, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
        RPY_CHECK(cudaMemcpyAsync(df, f_host, sizeof(double) * n3, cudaMemcpyHostToDevice, t.side_stream));
        RPY_CHECK(cudaEventRecord(t.h2d_ev, t.side_stream));
        RPY_TRY(rpy_tree_update_positions(h, dp, stream));
        RPY_CHECK(cudaStreamWaitEvent(st, t.h2d_ev, 0));
    } else {
        RPY_CHECK(cudaMemcpyAsync(df, f_host, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    }
    RPY_TRY(rpy_forest_matvec(h, df, s_host, du, stream));
    RPY_CHECK(cudaMemcpyAsync(u_host, du, sizeof(double) * n3, cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    return RPY_OK;
}

int rpy_forest_matvec(rpy_tree h, const double *f_dev, const double *s_host, double *u_dev, void *stream) {
    if (!valid(h) || !f_dev || !u_dev || !s_host) return RPY_ERR_INVALID;
    Tree &t = h->t;
    for (int k = 0; k < t.nsys; ++k)
        if (!std::isfinite(s_host[k])) return RPY_ERR_INVALID;
    DeviceGuard g(t.device);
    return run_matvec(t, f_dev, s_host, u_dev, RPY_PART_ALL, static_cast<cudaStream_t>(stream));
}

int rpy_matvec_parts(rpy_tree h, const double *f_dev, double s, double *u_dev, int parts, void *stream) {
    if (!valid(h) || !f_dev || !u_dev || !std::isfinite(s) || parts < 1 || parts > 3) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    std::vector<double> sv(t.nsys, s);
    return run_matvec(t, f_dev, sv.data(), u_dev, parts, static_cast<cudaStream_t>(stream));
}

int rpy_matvec(rpy_tree h, const double *f_dev, double s, double *u_dev, void *stream) {
    return rpy_matvec_parts(h, f_dev, s, u_dev, RPY_PART_ALL, stream);
}

int rpy_matvec_batched(rpy_tree const *trees, int ntrees, const double *const *f_dev, const double *kT_over_eta,
                       double *const *u_dev, void *stream) {
    if (!trees || ntrees < 0 || (ntrees > 0 && (!f_dev || !kT_over_eta || !u_dev))) return RPY_ERR_INVALID;
    for (int k = 0; k < ntrees; ++k)
        if (!valid(trees[k]) || !f_dev[k] || !u_dev[k] || !std::isfinite(kT_over_eta[k])) return RPY_ERR_INVALID;
    for (int k = 0; k < ntrees; ++k) RPY_TRY(rpy_matvec(trees[k], f_dev[k], kT_over_eta[k], u_dev[k], stream));
    return RPY_OK;
}

int rpy_matvec_oneshot(const double *pos_dev, int64_t n, double a, const double *f_dev, double s, int digits,
                       double *u_dev, void *stream) {
    if (!pos_dev || !f_dev || !u_dev || !std::isfinite(s)) return RPY_ERR_INVALID;
    rpy_tree t = nullptr;
    RPY_TRY(rpy_tree_build(pos_dev, n, a, digits, 0, RPY_FP64, stream, &t));
    int st = rpy_matvec(t, f_dev, s, u_dev, stream);
    if (st == RPY_OK) st = rpy_tree_sync(t);
    rpy_tree_free(t);
    return st;
}

int rpy_matvec_host(const double *pos_host, int64_t n, double a, const double *f_host, double s, int digits,
                    int precision, double *u_host, void *stream) {
    if (!pos_host || !f_host || !u_host || n < 1 || !std::isfinite(s)) return RPY_ERR_INVALID;
    RPY_TRY(have_device());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Tree scratch;
    double *d = nullptr;
    RPY_TRY(dev_alloc(scratch, (void **)&d, sizeof(double) * 9 * size_t(n)));
    double *dp = d, *df = d + 3 * n, *du = d + 6 * n;
    int rc = RPY_OK;
    rpy_tree t = nullptr;
    do {
        cudaError_t e = cudaMemcpyAsync(dp, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(df, f_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = check_cuda("h2d", e); break; }
        rc = rpy_tree_build(dp, n, a, digits, 0, precision, stream, &t);
        if (rc != RPY_OK) break;
        rc = rpy_matvec(t, df, s, du, stream);
        if (rc != RPY_OK) break;
        e = cudaMemcpyAsync(u_host, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = check_cuda("d2h", e);
    } while (0);
    if (t) rpy_tree_free(t);
    tree_release(scratch);
    return rc;
}

int rpy_evaluate(const double *src_pos_dev, const double *src_f_dev, int64_t ns, const double *tgt_pos_dev,
                 int64_t nt, double a, double s, const rpy_build_params *params, double *u_tgt_dev, void *stream) {
    if (!src_pos_dev || !src_f_dev || !tgt_pos_dev || !u_tgt_dev || !params || ns < 1 || nt < 1 ||
        !std::isfinite(s) || !(a > 0.0) || !std::isfinite(a))
        return RPY_ERR_INVALID;
    RPY_TRY(check_params(*params));
    RPY_TRY(have_device());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = ns + nt;
    Tree scratch;
    double *d = nullptr;
    RPY_TRY(dev_alloc(scratch, (void **)&d, sizeof(double) * 9 * size_t(n)));
    double *dp = d, *df = d + 3 * n, *du = d + 6 * n;
    int rc = RPY_OK;
    rpy_tree t = nullptr;
    do {
        // the union of sources and targets, targets as beads without force
        cudaError_t e = cudaMemcpyAsync(dp, src_pos_dev, sizeof(double) * 3 * ns, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp + 3 * ns, tgt_pos_dev, sizeof(double) * 3 * nt, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(df, src_f_dev, sizeof(double) * 3 * ns, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(df + 3 * ns, 0, sizeof(double) * 3 * nt, st);
        if (e != cudaSuccess) {
            rc = check_cuda("evaluate copies", e);
            break;
        }
        const int64_t off[2] = {0, n};
        rc = rpy_forest_build(dp, off, 1, &a, params, stream, &t);
        if (rc != RPY_OK) break;
        rc = rpy_forest_matvec(t, df, &s, du, stream);
        if (rc != RPY_OK) break;
        e = cudaMemcpyAsync(u_tgt_dev, du + 3 * ns, sizeof(double) * 3 * nt, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = check_cuda("evaluate", e);
    } while (0);
    if (t) rpy_tree_free(t);
    tree_release(scratch);
    return rc;
}

int rpy_laplace_far(rpy_tree h, const double *q_dev, double *out_dev, void *stream) {
    if (!valid(h) || !q_dev || !out_dev) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    return run_laplace_far(t, q_dev, out_dev, static_cast<cudaStream_t>(stream));
}

int rpy_tree_sync(rpy_tree h) {
    if (!valid(h)) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    cudaError_t e = wait_done(t);
    if (e != cudaSuccess) return check_cuda("sync", e);
    unsigned status = 0;
    RPY_CHECK(cudaMemcpy(&status, t.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (status & DEVERR_NONFINITE) return RPY_ERR_NONFINITE;
    if (status & DEVERR_TIMEOUT) return RPY_ERR_TIMEOUT;
    if (status) return RPY_ERR_INTERNAL;
    return RPY_OK;
}

int rpy_tree_export(rpy_tree h, int field, void *dst, int64_t capacity, int64_t *bytes_out) {
    if (!valid(h)) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    RPY_TRY(rpy_tree_sync(h));
    const void *src = nullptr;
    int64_t bytes = 0;
    switch (field) {
        case RPY_FIELD_PERM: src = t.perm; bytes = 4 * t.n; break;
        case RPY_FIELD_KEYS: src = t.keys; bytes = 8 * t.n; break;
        case RPY_FIELD_BOX_LEVEL: src = t.b_level; bytes = 4 * int64_t(t.nbox); break;
        case RPY_FIELD_BOX_RANGE: break;
        case RPY_FIELD_BOX_PARENT: src = t.b_parent; bytes = 4 * int64_t(t.nbox); break;
        case RPY_FIELD_BOX_CENTER: src = t.b_center; bytes = 24 * int64_t(t.nbox); break;
        case RPY_FIELD_BOX_LEAF: src = t.b_leaf; bytes = 4 * int64_t(t.nbox); break;
        case RPY_FIELD_BOX_SYS: src = t.b_sys; bytes = 4 * int64_t(t.nbox); break;
        case RPY_FIELD_BOX_SIDE: src = t.b_side; bytes = 8 * int64_t(t.nbox); break;
        case RPY_FIELD_LEAVES: src = t.leaves; bytes = 4 * int64_t(t.nleaf); break;
        case RPY_FIELD_U_OFF: src = t.u_off; bytes = 4 * int64_t(t.nleaf + 1); break;
        case RPY_FIELD_U_IDX: src = t.u_idx; bytes = 4 * t.n_u; break;
        case RPY_FIELD_W_OFF: src = t.w_off; bytes = 4 * int64_t(t.nleaf + 1); break;
        case RPY_FIELD_W_IDX: src = t.w_idx; bytes = 4 * t.n_w; break;
        case RPY_FIELD_X_OFF: src = t.x_off; bytes = 4 * int64_t(t.nbox + 1); break;
        case RPY_FIELD_X_IDX: src = t.x_idx; bytes = 4 * t.n_x; break;
        case RPY_FIELD_V_OFF:
        case RPY_FIELD_V_IDX:
            RPY_TRY(tree_build_vlists(t, nullptr));   // debug export: legacy stream, synchronous
            src = field == RPY_FIELD_V_OFF ? (const void *)t.v_off : (const void *)t.v_idx;
            bytes = field == RPY_FIELD_V_OFF ? 4 * int64_t(t.nbox + 1) : 4 * t.n_v;
            break;
        case RPY_FIELD_CUBE: src = t.sys_cube; bytes = 32 * int64_t(t.nsys); break;
        case RPY_FIELD_D_OFF: src = t.d_off; bytes = 4 * int64_t(t.nleaf + 1); break;
        case RPY_FIELD_D_IDX: src = t.d_idx; bytes = 4 * t.n_d; break;
        default: return RPY_ERR_INVALID;
    }
    if (field == RPY_FIELD_BOX_RANGE) bytes = 8 * int64_t(t.nbox);
    if (bytes_out) *bytes_out = bytes;
    if (!dst) return RPY_OK;
    if (capacity < bytes) return RPY_ERR_INVALID;
    if (field == RPY_FIELD_BOX_RANGE) {
        std::vector<int> b(t.nbox), e(t.nbox);
        RPY_CHECK(cudaMemcpy(b.data(), t.b_begin, 4 * size_t(t.nbox), cudaMemcpyDeviceToHost));
        RPY_CHECK(cudaMemcpy(e.data(), t.b_end, 4 * size_t(t.nbox), cudaMemcpyDeviceToHost));
        int *o = static_cast<int *>(dst);
        for (int i = 0; i < t.nbox; ++i) {
            o[2 * i] = b[i];
            o[2 * i + 1] = e[i];
        }
        return RPY_OK;
    }
    if (bytes) RPY_CHECK(cudaMemcpy(dst, src, size_t(bytes), cudaMemcpyDeviceToHost));
    return RPY_OK;
}

int rpy_tree_stats(rpy_tree h, rpy_stats *o) {
    if (!valid(h) || !o) return RPY_ERR_INVALID;
    RPY_TRY(rpy_tree_sync(h));
    Tree &t = h->t;
    std::memset(o, 0, sizeof(*o));
    o->n_beads = t.n;
    o->n_systems = t.nsys;
    o->n_boxes = t.nbox;
    o->n_leaves = t.nleaf;
    o->depth = t.nlevels - 1;
    o->order_p = t.p;
    o->exp_nodes = t.tabs ? t.tabs->s : 0;
    o->exp_terms = t.tabs ? 2 * t.tabs->S : 0;
    o->leaf_cap = t.params.leaf_cap;
    o->digits = t.params.digits;
    o->precision = t.params.precision;
    o->max_leaf_count = t.max_leaf_count;
    o->leaves_over_cap = t.leaves_over_cap;
    o->u_pairs = t.u_pairs;
    o->n_ulist = t.n_u;
    o->n_wlist = t.n_w;
    o->n_xlist = t.n_x;
    o->n_vpairs = t.n_v;
    o->n_dlist = t.n_d;
    o->d_pairs = t.d_pairs;
    o->device_bytes = t.device_bytes;
    o->build_ms = t.build_ms;
    o->quad = t.params.quad;
    return RPY_OK;
}

int rpy_tree_footprint(int64_t n, int digits, int precision, int leaf_cap, int64_t *bytes) {
    if (!bytes || n < 1 || (digits != 3 && digits != 6 && digits != 9)) return RPY_ERR_INVALID;
    if (leaf_cap <= 0) leaf_cap = default_leaf_cap(digits);
    const ExpQuad &q = exp_quadrature(digits);
    int p = default_order(digits);
    double es = precision == RPY_FP32 ? 8.0 : 16.0;
    // boxes: leaves ~ 2n/cap on clustered data, plus internal boxes (< leaves/7 * 8)
    double nbox = 4.0 * double(n) / double(leaf_cap) + 64.0;
    const int xf = plane_wave_frames(nbox, es, q.half());
    // M, L, plane waves, L2P scratch, and (rotation-based M2M) a per-octant share
    // slot for the boxes of one level, counted here for every box
    const double m2m = (precision != RPY_FP32 || p >= 12) ? 8.0 * kSets * ncoef(p) : 0.0;
    double per_box = es * (2.0 * kSets * ncoef(p) + 2.0 * 2 * xf * kSets * q.half() + 18.0 * ncoef(p) + m2m) +
                     4.0 * (8 + 27 + 3 + 12) + 32.0;
    double per_bead = 3 * 8 /*pos*/ + 8 /*key*/ + 4 + 4 + 9 * 8 /*fs, unear, ufar*/ + 27 * 4 /*U list share*/ +
                      (precision == RPY_FP32 ? 9 * 4 /*p32, f32*/ : 0);
    *bytes = int64_t(nbox * per_box + double(n) * per_bead + 32.0 * 1024 * 1024);
    return RPY_OK;
}

void rpy_tree_free(rpy_tree h) {
    if (!valid(h)) return;
    Tree &t = h->t;
    {
        DeviceGuard g(t.device);
        wait_done(t);
        tree_release(t);
        for (int k = 0; k < Tree::kMaxMarks; ++k)
            if (t.ev[k]) cudaEventDestroy(t.ev[k]);
        if (t.host_io) cudaFree(t.host_io);
        if (t.done) cudaEventDestroy(t.done);
        drop_graph(t);
        if (t.cap_stream) cudaStreamDestroy(t.cap_stream);
        if (t.side_stream) cudaStreamDestroy(t.side_stream);
        if (t.fork_ev) cudaEventDestroy(t.fork_ev);
        if (t.join_ev) cudaEventDestroy(t.join_ev);
        if (t.h2d_ev) cudaEventDestroy(t.h2d_ev);
    }
    h->magic = 0;
    delete h;
}

int rpy_tree_set_profiling(rpy_tree h, int enable) {
    if (!valid(h)) return RPY_ERR_INVALID;
    h->t.prof = enable != 0;
    return RPY_OK;
}

int rpy_tree_stage_times(rpy_tree h, double *ms, int n) {
    if (!valid(h) || !ms || n < 0) return RPY_ERR_INVALID;
    Tree &t = h->t;
    DeviceGuard g(t.device);
    RPY_CHECK(wait_done(t));
    for (int k = 0; k < n; ++k) ms[k] = 0.0;
    // each mark opens an interval of its stage that the next mark closes
    for (int i = 0; i + 1 < t.n_marks; ++i) {
        const int k = t.ev_stage[i];
        if (k >= RPY_NUM_STAGES || k >= n) continue;
        float v = 0.f;
        RPY_CHECK(cudaEventElapsedTime(&v, t.ev[i], t.ev[i + 1]));
        ms[k] += v;
    }
    return RPY_OK;
}

int64_t rpy_launch_count(void) { return g_launches.load(); }

int rpy_debug_wait_timeout(double limit_ms, void *stream) {
    if (!(limit_ms > 0.0) || limit_ms > 2000.0) return RPY_ERR_INVALID;
    RPY_TRY(have_device());
    return wait_selftest(limit_ms, static_cast<cudaStream_t>(stream));
}

int rpy_bounding_cube_noalloc(const double *pos_dev, int64_t n, double *cube_dev, void *stream) {
    if (!pos_dev || !cube_dev) {
        set_last_error("rpy_bounding_cube_noalloc: pos_dev and cube_dev must be device pointers, not NULL");
        return RPY_ERR_INVALID;
    }
    if (n < 1) {
        set_last_error("rpy_bounding_cube_noalloc: n must be at least 1");
        return RPY_ERR_INVALID;
    }
    RPY_TRY(have_device());
    return bounding_cube_noalloc(pos_dev, n, cube_dev, static_cast<cudaStream_t>(stream));
}

int rpy_alu_peak(int precision, double *flops_per_s, void *stream) {
    if (!flops_per_s || (precision != RPY_FP64 && precision != RPY_FP32)) return RPY_ERR_INVALID;
    RPY_TRY(have_device());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    RPY_CHECK(cudaGetDevice(&dev));
    RPY_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int blocks = sms * 8, threads = 256;
    int iters = precision == RPY_FP64 ? 2048 : 65536;
    Tree scratch;
    void *buf = nullptr;
    RPY_TRY(dev_alloc(scratch, &buf, sizeof(double) * size_t(blocks) * threads));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (precision == RPY_FP64)
            k_fma_probe<double><<<blocks, threads, 0, st>>>(static_cast<double *>(buf), iters, 0.999999, 1e-7);
        else
            k_fma_probe<float><<<blocks, threads, 0, st>>>(static_cast<float *>(buf), iters, 0.9999f, 1e-4f);
        RPY_LAUNCHED(1);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            tree_release(scratch);
            return check_cuda("alu probe", e);
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tree_release(scratch);
    *flops_per_s = 2.0 * 8.0 * double(iters) * blocks * threads / (best * 1e-3);
    return RPY_OK;
}

int rpy_debug_table(int p, int digits, int which, double *dst, int64_t capacity, int64_t *count) {
    if (p < 2 || p > kMaxP || ((digits < 3 || digits > 6) && digits != 9)) return RPY_ERR_INVALID;
    OpTables *h = nullptr;
    RPY_TRY(host_tables(p, digits, &h));
    std::vector<double> tmp;
    const std::vector<double> *v = nullptr;
    switch (which) {
        case 1: v = &h->m2m_t; break;
        case 2: v = &h->l2l_t; break;
        case 3: v = &h->rot_fwd; break;
        case 4: v = &h->rot_bwd; break;
        case 5: v = &h->m2x_c; break;
        case 6: v = &h->x2l_c; break;
        case 7:   // stored plane waves: k, cos, sin, w/M per entry
            for (int e = 0; e < h->S; ++e) {
                tmp.push_back(h->e_k[e]);
                tmp.push_back(h->e_cos[e]);
                tmp.push_back(h->e_sin[e]);
                tmp.push_back(h->e_wm[e]);
            }
            v = &tmp;
            break;
        case 8: v = &h->shift; break;
        case 9:   // groups: per direction: ngroups, then per group (mask, nslots, slot|shift<<8 ...)
            for (int d = 0; d < kDirs; ++d) {
                int ng = h->grp_n[d];
                tmp.push_back(ng);
                for (int g = 0; g < ng; ++g) {
                    int a = h->grp_off[d * (kGroupMax + 1) + g], b = h->grp_off[d * (kGroupMax + 1) + g + 1];
                    tmp.push_back(h->grp_mask[d * kGroupMax + g]);
                    tmp.push_back(b - a);
                    for (int z = a; z < b; ++z) tmp.push_back(h->slot_list[d * 216 + z]);
                }
                for (int c = 0; c < 8; ++c) tmp.push_back(h->child_shift[d * 8 + c]);
            }
            v = &tmp;
            break;
        case 10:   // rotation block offsets
            for (int o : h->rot_off) tmp.push_back(o);
            v = &tmp;
            break;
        case 12: v = &h->orot_fwd; break;
        case 13: v = &h->orot_bwd; break;
        case 14: v = &h->zm2m; break;
        case 15: v = &h->zl2l; break;
        case 16: v = &h->shz; break;
        case 17: v = &h->shx; break;
        case 18: v = &h->shy; break;
        case 11:   // quadrature: s, then lambda, weight, M per node
        {
            const ExpQuad &q = exp_quadrature(digits);
            tmp.push_back(q.s);
            for (int k = 0; k < q.s; ++k) {
                tmp.push_back(q.lambda[k]);
                tmp.push_back(q.weight[k]);
                tmp.push_back(q.m[k]);
            }
            v = &tmp;
            break;
        }
        default: return RPY_ERR_INVALID;
    }
    if (count) *count = int64_t(v->size());
    if (!dst) return RPY_OK;
    if (capacity < int64_t(v->size())) return RPY_ERR_INVALID;
    std::memcpy(dst, v->data(), sizeof(double) * v->size());
    return RPY_OK;
}

}  // extern "C"
