// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "../../include/rpyfmm.h"

#define RPY_HD __host__ __device__ __forceinline__

namespace rpy {

// ---------------------------------------------------------------- status

// Device-side error flags (bitwise OR into DevStatus::flags).
enum : unsigned {
    DEVERR_NONFINITE = 1u,     // a position was NaN/inf
    DEVERR_STACK = 2u,         // list-builder traversal stack overflow
    DEVERR_CAPACITY = 4u,      // a fixed-size device table overflowed
    DEVERR_TIMEOUT = 8u,       // a bounded device wait (an mbarrier of a bulk-copy pipeline) gave up
};

struct CudaError {
    cudaError_t err;
    const char *what;
};

void set_last_cuda_error(const char *what, cudaError_t e);
void set_last_error(const char *msg);
int bounding_cube_noalloc(const double *pos_dev, int64_t n, double *cube_dev, cudaStream_t st);
int check_cuda(const char *what, cudaError_t e);   // returns RPY_OK or RPY_ERR_CUDA/OOM

#define RPY_CHECK(call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return rpy::check_cuda(#call, e_);         \
    } while (0)

#define RPY_TRY(expr)                                                     \
    do {                                                                  \
        int s_ = (expr);                                                  \
        if (s_ != RPY_OK) return s_;                                      \
    } while (0)

// ---------------------------------------------------------------- complex

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T x, y;
};

template <typename T> RPY_HD cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> RPY_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> RPY_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> RPY_HD cpx<T> operator*(cpx<T> a, cpx<T> b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename T> RPY_HD cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T> RPY_HD cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T> RPY_HD void operator+=(cpx<T> &a, cpx<T> b) { a.x += b.x; a.y += b.y; }
// multiply by i^k
template <typename T> RPY_HD cpx<T> mul_ipow(cpx<T> a, int k) {
    switch (k & 3) {
        case 0: return a;
        case 1: return mk(-a.y, a.x);
        case 2: return mk(-a.x, -a.y);
        default: return mk(a.y, -a.x);
    }
}

// index of coefficient (n, m), 0 <= m <= n, in triangular storage
RPY_HD int tri(int n, int m) { return n * (n + 1) / 2 + m; }
RPY_HD int ncoef(int p) { return (p + 1) * (p + 2) / 2; }

// ---------------------------------------------------------------- settings

constexpr int kSets = 4;          // Laplace charge sets L1..L4 (Sec. 2)
constexpr int kDirs = 6;          // +z -z +x -x +y -y plane-wave directions
// Plane-wave frames handled per M2X / X2X / X2L pass: all three while the
// outgoing and incoming buffers of six directions take at most kXAllFramesBytes,
// else one frame (two directions) per pass, which needs a third of the memory.
constexpr double kXAllFramesBytes = 64e9;
inline int plane_wave_frames(double nbox, double elem_bytes, int S) {
    return 2.0 * nbox * kDirs * 4 * double(S) * elem_bytes <= kXAllFramesBytes ? 3 : 1;
}
constexpr int kMaxP = 29;         // largest supported expansion order (p + 2 < 32 warp lanes)
constexpr int kMaxLevel = 21;
constexpr int kItemTargets = 256;   // targets per near-field work item

struct ExpQuad {                  // plane-wave quadrature (box units)
    int s = 0;                    // lambda nodes
    std::vector<double> lambda, weight;
    std::vector<int> m;           // trapezoid counts (even)
    int terms() const { int t = 0; for (int v : m) t += v; return t; }
    int half() const { return terms() / 2; }
};

const ExpQuad &exp_quadrature(int digits);
int default_order(int digits);
int default_leaf_cap(int digits);

// Operator tables of one (p, digits) setting, uploaded once per device.
struct OpTables {
    int p = 0, nc = 0, digits = 0, s = 0, S = 0;   // S = stored plane waves (half of sum M_k)
    // host copies (double) ----------------------------------------------
    std::vector<double> m2m_t;    // [8][D][D] transposed real M2M (D = 2 nc), column = output
    std::vector<double> l2l_t;    // [8][D][D] transposed real L2L
    std::vector<double> rot_fwd;  // [2 frames][sum_n (2n+1)^2] real blocks world -> frame (x, y)
    std::vector<double> rot_bwd;  // [2 frames][...] frame -> world
    std::vector<int> rot_off;     // [p+1] offset of degree-n block
    std::vector<double> m2x_c;    // [s][nc]  lambda_k^n / sqrt((n-m)!(n+m)!)
    std::vector<double> x2l_c;    // [s][nc]  (-lambda_k)^n / sqrt((n-m)!(n+m)!)
    std::vector<int> e_k;         // [S] node of stored plane wave e
    std::vector<double> e_cos, e_sin, e_wm;   // [S] cos a, sin a, w_k / M_k
    std::vector<int> k_start;     // [s+1] first stored e of node k
    // wave pairs: stored waves j and M_k/2 - j of a node have angles a and pi - a,
    // so one set of products serves both; unit t of node k holds wave t and, for
    // 0 < t < M_k/2 - t, its partner M_k/2 - t
    std::vector<int> u_k;         // [NU] node of unit u
    std::vector<int> u_start;     // [s+1] first unit of node k
    std::vector<double> shift;    // [216][S][2] e^{-lambda dz + i lambda (dx cos a + dy sin a)}
    // the same shifts per axis: shift(off) = shz[iz] * shx[ix] * shy[iy] with
    // off = ix + 6 iy + 36 iz (offset d = index - 2.5 along each axis)
    std::vector<double> shz;      // [6][S] e^{-lambda dz}
    std::vector<double> shx, shy; // [6][S][2] e^{i lambda dx cos a}, e^{i lambda dy sin a}
    // merge-and-shift groups per direction
    std::vector<int> grp_off;     // [6][G_MAX+1] start of group g in slot list (per direction)
    std::vector<int> grp_n;       // [6] number of groups
    std::vector<int> grp_mask;    // [6][G_MAX] child mask of group
    std::vector<int> slot_list;   // [6][216] (slot | (shift index << 8)) by group
    std::vector<int> child_shift; // [6][8] shift index parent centre -> child centre
    std::vector<double> roots;    // [2S][2] e^{2 pi i r / M_k}, r < M_k, node k at 2 k_start[k]
    std::vector<double> rec_a, rec_b, rec_c, rec_cm;   // harmonic recurrences to degree p + 2
    // ladder coefficients of the derivative expansions, index tri(k, m), degree <= p + 2:
    // local:     lz = sqrt((k+1+m)(k+1-m)), lp = sqrt((k-m+1)(k-m+2)), lq = sqrt((k+m+1)(k+m+2))
    // multipole: mz = sqrt((k+m)(k-m)),     mp = sqrt((k+m)(k+m-1)),   mq = sqrt((k-m)(k-m-1))
    std::vector<double> lad;      // [6][ncoef(p+2)] in the order lz lp lq mz mp mq
    // rotation-based M2M / L2L: per child octant, rotations world -> frame whose z axis is
    // the shift direction and back, and the m-diagonal z-shift coefficients
    std::vector<double> orot_fwd, orot_bwd;   // [8][rot_len]
    // the same rotations factored through z-y-z Euler angles (layout in rpy_tables.cu)
    std::vector<double> frot_fwd, frot_bwd;   // [2 frames][frot_len]
    std::vector<double> forot_fwd, forot_bwd; // [8 octants][frot_len]
    std::vector<int> frot_off;                // [p+2] offset of degree n
    std::vector<double> zm2m, zl2l;           // [ncoef(p)][p+1]: output (n,m), input degree k
};
constexpr int kGroupMax = 32;

int build_tables(int p, int digits, OpTables &t);   // host computation, no CUDA

// device copies
template <typename T>
struct DevTables {
    int p, nc, s, S, rot_len;
    const T *m2m_t, *l2l_t, *rot_fwd, *rot_bwd;
    const int *rot_off;
    const T *rec_a, *rec_b, *rec_c, *rec_cm;
    const T *lad;
    const T *orot_fwd, *orot_bwd, *zm2m, *zl2l;
    const T *frot_fwd, *frot_bwd, *forot_fwd, *forot_bwd;
    const int *frot_off;
    int frot_len;
    const cpx<T> *roots;
    const T *m2x_c, *x2l_c;
    const int *e_k, *k_start;
    const int *u_k, *u_start;   // wave-pair units
    int NU;
    const T *e_cos, *e_sin, *e_wm;
    const cpx<T> *shift;
    const cpx<T> *shiftp;   // the same rows with stride Sp (S rounded up to even: 16-byte rows for bulk copies)
    int Sp;
    const T *shz;
    const cpx<T> *shx, *shy;
    const int *grp_off, *grp_n, *grp_mask, *slot_list, *child_shift;
};

// ---------------------------------------------------------------- tree

// Per-system constants of the pair formulas and of Eq. (2.8), formed once per
// change of kT/eta (the kernels then do no FP64 division of their own).
struct PairConst {
    double a, co, cf, k23, nk2;   // co = s/(6 pi a), cf = s/(8 pi), k23 = 2a^2/3, nk2 = -2a^2
    double a2x4;                  // 4a^2
    double C1, C2, icube;         // C1 = s/(8 pi), C2 = s a^2/(12 pi), 1/(side of the root cube)
    float f_a2x4, f_tiny2, f_k23, f_nk2;   // FP32 copies; tiny2 = 1e-6 a^2
    float f_co_cf, f_nco_c9, f_co_c3, f_pad;   // co/cf, -(co/cf) 9/(32a), (co/cf) 3/(32a)
};

struct Tree {
    int device = 0;
    bool built = false;               // false while (or after a failed) build
    cudaStream_t last_stream = nullptr;
    int64_t n = 0;
    int nsys = 0;
    rpy_build_params params{};
    int p = 0;
    std::vector<int64_t> sys_off_h;   // host copy, nsys+1
    std::vector<double> a_h;          // host copy, nsys
    // systems (device)
    int64_t *sys_off = nullptr;
    double *sys_a = nullptr;
    double *sys_cube = nullptr;       // [nsys][4]: centre x, y, z, side
    // beads (device, sorted order)
    int *perm = nullptr;              // sorted -> caller
    uint64_t *keys = nullptr;
    double *pos = nullptr;            // SoA [3][n]
    int *bead_sys = nullptr;
    // boxes (device)
    int nbox = 0, nbox_cap = 0, nlevels = 0;
    std::vector<int> level_off;       // host, nlevels+1
    int *b_level = nullptr, *b_begin = nullptr, *b_end = nullptr, *b_parent = nullptr;
    int *b_child = nullptr;           // [nbox][8]
    int *b_coll = nullptr;            // [nbox][27]
    int *b_cell = nullptr;            // [nbox][3]
    int *b_sys = nullptr, *b_leaf = nullptr, *b_leafid = nullptr;
    double *b_center = nullptr;       // [nbox][3]
    double *b_side = nullptr;
    int nleaf = 0;
    int *leaves = nullptr;
    int *bead_leaf = nullptr;         // [n] leaf index of each sorted bead
    // lists (device CSR)
    int *u_off = nullptr, *u_idx = nullptr;
    int *w_off = nullptr, *w_idx = nullptr;
    int *x_off = nullptr, *x_idx = nullptr;
    int64_t n_u = 0, n_w = 0, n_x = 0, u_pairs = 0;
    int max_leaf_count = 0, leaves_over_cap = 0;
    // level-2+ boxes with children (X2X parents), and boxes at level >= 2
    int n_x2x_par = 0, *x2x_par = nullptr;
    // direct (P2P) substitutes for small W and X interactions, per leaf
    int *d_off = nullptr, *d_idx = nullptr;
    // near-field work items (leaf, first target) of at most kItemTargets targets, in
    // decreasing cost order for the U-list pass and for the direct-substitute pass
    int n_items = 0;
    int2 *u_items = nullptr, *d_items = nullptr;
    // the near list of the full matvec: per leaf the U list, then the direct substitutes;
    // its work items in decreasing cost order (one pass for both)
    int *m_off = nullptr, *m_idx = nullptr;
    int2 *m_items = nullptr;
    int64_t n_d = 0, d_pairs = 0;
    int direct_w = 0, direct_x = 0;    // bead-count thresholds in use (0 = none)
    // expansions and matvec workspace
    void *M = nullptr, *L = nullptr, *Xo = nullptr, *Xi = nullptr;
    int x_frames = 3;                 // plane-wave frames per pass (3 or 1)
    void *m2m_scratch = nullptr;      // FP64 M2M: [boxes of the widest level][8 octants][4][nc] child shares
    void *EVg = nullptr;              // [nleaf][18][ncoef(p)] derived local expansions of Eq. (2.8)
    double *fs = nullptr;             // sorted forces SoA [3][n]
    float *p32 = nullptr;             // FP32 form: sorted positions as hi + lo floats, [6][n] (x,y,z hi; x,y,z lo)
    float *f32 = nullptr;             // FP32 form: sorted forces [3][n]
    double *u_near = nullptr, *u_far = nullptr, *u_dir = nullptr;   // sorted [n][3]
    double *host_io = nullptr;        // rpy_tree_matvec_host: positions, forces, velocities [9][n] (caller order),
                                      // allocated on its first call, kept across rebuilds
    double *lap_q = nullptr;          // [n][4] sorted charges for the Laplace debug path
    double *sys_s = nullptr;          // [nsys] kT/eta of the last matvec
    PairConst *sys_pc = nullptr;      // [nsys] constants derived from a, kT/eta and the root cube
    std::vector<double> sys_s_h;
    unsigned *dev_status = nullptr;
    int64_t device_bytes = 0;
    double build_ms = 0;
    // debug V lists (built on request)
    int *v_off = nullptr, *v_idx = nullptr;
    int64_t n_v = 0;
    // tables
    const OpTables *tabs = nullptr;   // the cached host tables of (p, quadrature rule); never freed
    void *dtabs_mem = nullptr;        // one device block holding all tables
    DevTables<double> dt64{};
    DevTables<float> dt32{};
    // device memory: blocks in use, and free blocks kept for the next rebuild
    struct Block {
        void *p;
        size_t bytes;
    };
    std::vector<Block> allocs;
    std::multimap<size_t, void *> cache;
    Tree *owner = nullptr;            // scratch trees take from and return to their owner's cache
    // per-stage profiling (events recorded between stages when enabled)
    bool prof = false;
    cudaEvent_t done = nullptr;       // recorded after every asynchronous call (survives the caller's stream)
    // CUDA graph of the matvec body (P2P .. L2P), captured on the second matvec of a build
    cudaStream_t cap_stream = nullptr;
    // captured matvec: the near field runs on side_stream beside the far field
    // (fork_ev / join_ev order the two branches inside the graph)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaEvent_t h2d_ev = nullptr;     // host-buffer step: the forces' copy (on side_stream) has landed
    cudaGraphExec_t gexec = nullptr;
    int matvecs = 0;                  // matvecs since the last build
    // stage marks of the last profiled matvec: event k opens an interval of stage
    // ev_stage[k] that the next mark closes (a stage may recur, e.g. once per plane-wave frame)
    static constexpr int kMaxMarks = 32;
    cudaEvent_t ev[kMaxMarks] = {};
    int ev_stage[kMaxMarks] = {};
    int n_marks = 0;
};

// stage markers: record event k on st when profiling is on
void prof_mark(Tree &t, int k, cudaStream_t st);

// count of kernel launches issued by the library
void note_launches(int n);
#define RPY_LAUNCHED(n) rpy::note_launches(n)

int tree_build(Tree &t, const double *pos_dev, cudaStream_t st);
int tree_alloc_workspace(Tree &t, cudaStream_t st);
int tree_upload_tables(Tree &t, cudaStream_t st);
int tree_build_vlists(Tree &t, cudaStream_t st);
void tree_release(Tree &t);     // owner: free everything; scratch: return blocks to the owner
void tree_recycle(Tree &t);     // move every block in use into the cache
int dev_alloc(Tree &t, void **p, size_t bytes);

// per-system constants seen by the kernels
struct SysConst {
    const double *cube;   // [nsys][4]
    const double *a;      // [nsys]
    const double *s;      // [nsys] kT/eta
    const PairConst *pc;  // [nsys]
};

// 2^l as a double, by its bit pattern (0 <= l < 1000)
__device__ __forceinline__ double pow2i(int l) { return __hiloint2double((1023 + l) << 20, 0); }

template <typename T>
int run_far_t(Tree &t, const DevTables<T> &D, const double *fs, const double *lapq, double *ufar, double *lapout,
              const SysConst &sc, cudaStream_t st);
// the polynomial (Cartesian Taylor) far field of RPY_FLAG_CARTESIAN trees (rpy_cart.cu)
template <typename T>
int run_cart_t(Tree &t, const double *fs, double *ufar, const SysConst &sc, cudaStream_t st);
int cart_terms(int P);   // monomials of total degree <= P
int wait_selftest(double limit_ms, cudaStream_t st);   // bounded mbarrier wait that must time out
constexpr int kCartMaxP = 10, kCartDefaultP = 8;
constexpr int kListU = 0, kListD = 1, kListM = 2;   // near list: U, direct substitutes, both
int run_p2p(Tree &t, const double *fs, double *out, const SysConst &sc, cudaStream_t st, int list);
int split_positions_f32(Tree &t, cudaStream_t st);
// the tree of a valid handle, else nullptr
Tree *tree_of(rpy_tree h);

// Makes `dev` current for the scope, restoring the caller's device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

const char *last_cuda_error_text();

// matvec stages (rpy_fmm.cu / rpy_p2p.cu)
int run_matvec(Tree &t, const double *f_dev, const double *s_per_sys_host, double *u_dev, int parts,
               cudaStream_t st);
int run_laplace_far(Tree &t, const double *q_dev, double *out_dev, cudaStream_t st);

// generic device helpers (rpy_tree.cu)
int exclusive_scan_i32(const int *in, int *out, int n, int *total_host, void *tmp, size_t tmp_bytes,
                       cudaStream_t st);
size_t scan_tmp_bytes(int n);

}  // namespace rpy
