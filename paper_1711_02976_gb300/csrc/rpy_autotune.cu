// Parameter search for the matvec (plane-wave quadrature rule, expansion
// order p, leaf capacity and the direct-substitution thresholds of small W / X
// interactions), and the FP64 direct sum on sampled targets that it measures
// accuracy against.
//
// The accuracy of the FMM at a setting is estimated, not assumed: the tuner
// draws K targets, sums RPY over all beads of their systems directly on the
// GPU in FP64 (the definition of Sec. 1: self term, r >= 2a branch, r < 2a
// overlap branch, coincident beads), and compares the matvec there.  For each
// candidate quadrature rule the order p is the smallest that keeps the sampled
// relative L2 error under margin x bound (bound 1e-3 or 1e-6 for 3 or 6
// digits), and the fastest (rule, p) pair is kept; leaf capacity and
// the direct-substitution thresholds are then chosen by timed matvecs
// (CUDA events on the caller's stream) among the settings that still meet it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <set>
#include <vector>

#include "rpy_internal.h"

namespace rpy {

constexpr double kPiT = 3.14159265358979323846;
constexpr int kDirThreads = 256;
constexpr int64_t kDirChunk = 32768;   // sources per CTA of the sampled direct sum

// One CTA per (sampled target, chunk of its system's sources): FP64 sum of
// D_tj F_j over the chunk; the self term belongs to the chunk holding t.
__global__ void k_direct_sampled(const double *pos, const double *f, const int64_t *tgt, const int64_t *sb,
                                 const int64_t *se, const double *av, const double *sv, int nchunk, double *part) {
    __shared__ double red[3][kDirThreads];
    const int k = blockIdx.x, c = blockIdx.y;
    const int64_t t = tgt[k];
    const double a = av[k], s = sv[k];
    const double co = s / (6.0 * kPiT * a), cf = s / (8.0 * kPiT);
    const double xt = pos[3 * t], yt = pos[3 * t + 1], zt = pos[3 * t + 2];
    const int64_t j0 = sb[k] + int64_t(c) * kDirChunk, j1 = min(se[k], j0 + kDirChunk);
    double ux = 0, uy = 0, uz = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const double fx = f[3 * j], fy = f[3 * j + 1], fz = f[3 * j + 2];
        if (j == t) {
            ux += co * fx;
            uy += co * fy;
            uz += co * fz;
            continue;
        }
        const double dx = xt - pos[3 * j], dy = yt - pos[3 * j + 1], dz = zt - pos[3 * j + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double RF = dx * fx + dy * fy + dz * fz;
        double t1, t2;
        if (r2 >= 4.0 * a * a) {
            const double r = sqrt(r2);
            t1 = cf / r * (1.0 + 2.0 * a * a / (3.0 * r2));
            t2 = cf / r * (1.0 - 2.0 * a * a / r2) / r2 * RF;
        } else if (r2 > 0.0) {
            const double r = sqrt(r2);
            t1 = co * (1.0 - 9.0 * r / (32.0 * a));
            t2 = co * 3.0 / (32.0 * a * r) * RF;
        } else {
            t1 = co;
            t2 = 0.0;
        }
        ux += t1 * fx + t2 * dx;
        uy += t1 * fy + t2 * dy;
        uz += t1 * fz + t2 * dz;
    }
    red[0][threadIdx.x] = ux;
    red[1][threadIdx.x] = uy;
    red[2][threadIdx.x] = uz;
    __syncthreads();
    for (int h = kDirThreads / 2; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h)
            for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[(size_t(k) * nchunk + c) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_gather_rows(const double *u, const int64_t *tgt, int64_t nt, double *out) {
    int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    for (int d = 0; d < 3; ++d) out[3 * k + d] = u[3 * tgt[k] + d];
}

namespace {

// Device scratch of one tuning run (allocated once, freed on every exit path).
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
};

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Sampled {
    std::vector<int64_t> tgt, sb, se;
    std::vector<double> a, s;
};

int check_forest_args(const double *pos_dev, const int64_t *off, int nsys, const double *a_host, const double *f_dev,
                      const double *s_host) {
    if (!pos_dev || !off || nsys < 1 || !a_host || !f_dev || !s_host) return RPY_ERR_INVALID;
    if (off[0] != 0) return RPY_ERR_INVALID;
    for (int k = 0; k < nsys; ++k) {
        if (off[k + 1] <= off[k]) return RPY_ERR_INVALID;
        if (!(a_host[k] > 0.0) || !std::isfinite(a_host[k]) || !std::isfinite(s_host[k])) return RPY_ERR_INVALID;
    }
    return RPY_OK;
}

Sampled describe(const int64_t *off, int nsys, const double *a_host, const double *s_host,
                 const std::vector<int64_t> &tg) {
    Sampled S;
    for (int64_t t : tg) {
        int k = int(std::upper_bound(off, off + nsys + 1, t) - off) - 1;
        S.tgt.push_back(t);
        S.sb.push_back(off[k]);
        S.se.push_back(off[k + 1]);
        S.a.push_back(a_host[k]);
        S.s.push_back(s_host[k]);
    }
    return S;
}

// FP64 direct sum at the sampled targets; u_host [nt][3].
int direct_sampled(const double *pos_dev, const double *f_dev, const Sampled &S, double *u_host, cudaStream_t st) {
    const int64_t nt = int64_t(S.tgt.size());
    if (nt == 0) return RPY_OK;
    int64_t maxlen = 0;
    for (int64_t k = 0; k < nt; ++k) maxlen = std::max(maxlen, S.se[k] - S.sb[k]);
    const int nchunk = int((maxlen + kDirChunk - 1) / kDirChunk);
    if (nt > 65535 * 16 || nchunk > 65535) return RPY_ERR_INVALID;
    Scratch sc;
    int64_t *dt = nullptr, *db = nullptr, *de = nullptr;
    double *da = nullptr, *ds = nullptr, *dp = nullptr;
    RPY_CHECK(sc.alloc(&dt, nt));
    RPY_CHECK(sc.alloc(&db, nt));
    RPY_CHECK(sc.alloc(&de, nt));
    RPY_CHECK(sc.alloc(&da, nt));
    RPY_CHECK(sc.alloc(&ds, nt));
    RPY_CHECK(sc.alloc(&dp, size_t(nt) * nchunk * 3));
    RPY_CHECK(cudaMemcpyAsync(dt, S.tgt.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(db, S.sb.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(de, S.se.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(da, S.a.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, st));
    RPY_CHECK(cudaMemcpyAsync(ds, S.s.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, st));
    // chunks past a short system's end write zero partials
    RPY_CHECK(cudaMemsetAsync(dp, 0, sizeof(double) * size_t(nt) * nchunk * 3, st));
    k_direct_sampled<<<dim3(unsigned(nt), unsigned(nchunk)), kDirThreads, 0, st>>>(pos_dev, f_dev, dt, db, de, da, ds,
                                                                                   nchunk, dp);
    RPY_LAUNCHED(1);
    RPY_CHECK(cudaGetLastError());
    std::vector<double> part(size_t(nt) * nchunk * 3);
    RPY_CHECK(cudaMemcpyAsync(part.data(), dp, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
    RPY_CHECK(cudaStreamSynchronize(st));
    for (int64_t k = 0; k < nt; ++k)
        for (int d = 0; d < 3; ++d) {
            double v = 0.0;
            for (int c = 0; c < nchunk; ++c) v += part[(size_t(k) * nchunk + c) * 3 + d];
            u_host[3 * k + d] = v;
        }
    return RPY_OK;
}

struct Trial {
    rpy_build_params prm;
    double err = INFINITY, ms = -1.0;
    int status = RPY_OK;
};

}  // namespace
}  // namespace rpy

using namespace rpy;

extern "C" int rpy_direct_sampled(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                                  const double *f_dev, const double *kT_over_eta_host, const int64_t *targets_host,
                                  int64_t nt, double *u_host, void *stream) {
    int s = check_forest_args(pos_dev, sys_offsets, nsys, a_host, f_dev, kT_over_eta_host);
    if (s != RPY_OK) return s;
    if (nt < 0 || (nt > 0 && (!targets_host || !u_host))) return RPY_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return RPY_ERR_NODEVICE;
    const int64_t N = sys_offsets[nsys];
    std::vector<int64_t> tg(targets_host, targets_host + nt);
    for (int64_t t : tg)
        if (t < 0 || t >= N) return RPY_ERR_INVALID;
    Sampled S = describe(sys_offsets, nsys, a_host, kT_over_eta_host, tg);
    return direct_sampled(pos_dev, f_dev, S, u_host, static_cast<cudaStream_t>(stream));
}

extern "C" int rpy_autotune(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                            const double *f_dev, const double *kT_over_eta_host, int digits, int precision,
                            const rpy_autotune_params *params, rpy_autotune_result *out, void *stream) {
    int s = check_forest_args(pos_dev, sys_offsets, nsys, a_host, f_dev, kT_over_eta_host);
    if (s != RPY_OK) return s;
    if (!out) return RPY_ERR_INVALID;
    if (digits != 3 && digits != 6 && digits != 9) return RPY_ERR_DIGITS;
    if (precision != RPY_FP64 && precision != RPY_FP32) return RPY_ERR_INVALID;
    if (digits == 9 && precision != RPY_FP64) return RPY_ERR_DIGITS;
    rpy_autotune_params P{};
    if (params) P = *params;
    if (P.n_samples < 0 || P.timed_reps < 0 || !(P.margin >= 0.0) || P.margin > 1.0) return RPY_ERR_INVALID;
    const int K0 = P.n_samples ? P.n_samples : 256;
    const double margin = P.margin > 0.0 ? P.margin : 0.3;
    const int reps = P.timed_reps ? P.timed_reps : 3;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return RPY_ERR_NODEVICE;
    auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *out = rpy_autotune_result{};

    const int64_t N = sys_offsets[nsys];
    Scratch sc;
    double *u = nullptr;
    RPY_CHECK(sc.alloc(&u, size_t(N) * 3));
    // a sample of targets with its FP64 direct sum and the device buffers that gather
    // the matvec's velocities there
    struct Probe {
        std::vector<int64_t> tg;
        std::vector<double> ref, got;
        double rn = 0.0;
        int64_t *dt = nullptr;
        double *ug = nullptr;
    };
    auto make_probe = [&](std::vector<int64_t> tgv, Probe &pr) -> int {
        pr.tg = std::move(tgv);
        const int64_t k = int64_t(pr.tg.size());
        pr.ref.assign(3 * k, 0.0);
        pr.got.assign(3 * k, 0.0);
        Sampled S = describe(sys_offsets, nsys, a_host, kT_over_eta_host, pr.tg);
        RPY_TRY(direct_sampled(pos_dev, f_dev, S, pr.ref.data(), st));
        pr.rn = 0.0;
        for (double v : pr.ref) pr.rn += v * v;
        RPY_CHECK(sc.alloc(&pr.ug, size_t(k) * 3));
        RPY_CHECK(sc.alloc(&pr.dt, size_t(k)));
        RPY_CHECK(cudaMemcpyAsync(pr.dt, pr.tg.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, st));
        return RPY_OK;
    };
    // sampled targets of the search (distinct, uniform over all beads)
    const int64_t K = std::min<int64_t>(K0, N);
    uint64_t seed = P.seed ? P.seed : 0x5EEDF00Dull;
    Probe probe;
    {
        std::set<int64_t> pick;
        while (int64_t(pick.size()) < K) pick.insert(int64_t(splitmix64(seed) % uint64_t(N)));
        RPY_TRY(make_probe(std::vector<int64_t>(pick.begin(), pick.end()), probe));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RPY_CHECK(cudaEventCreate(&e0));
    RPY_CHECK(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } evg{e0, e1};

    const double bound = digits == 3 ? 1e-3 : (digits == 6 ? 1e-6 : 1e-9);
    const double goal = margin * bound;
    std::vector<Trial> trials;

    // one trial: build, one untimed matvec, the sampled error on `pr`, optionally `reps`
    // timed matvecs
    auto run = [&](rpy_build_params prm, bool timed, Trial &T, Probe &pr) -> int {
        T.prm = prm;
        rpy_tree tree = nullptr;
        int r = rpy_forest_build(pos_dev, sys_offsets, nsys, a_host, &prm, stream, &tree);
        if (r != RPY_OK) {
            T.status = r;
            return r;
        }
        struct TreeGuard {
            rpy_tree t;
            ~TreeGuard() { rpy_tree_free(t); }
        } tgd{tree};
        r = rpy_forest_matvec(tree, f_dev, kT_over_eta_host, u, stream);
        if (r != RPY_OK) {
            T.status = r;
            return r;
        }
        const int64_t k = int64_t(pr.tg.size());
        k_gather_rows<<<unsigned((k + 127) / 128), 128, 0, st>>>(u, pr.dt, k, pr.ug);
        RPY_LAUNCHED(1);
        RPY_CHECK(cudaGetLastError());
        RPY_CHECK(cudaMemcpyAsync(pr.got.data(), pr.ug, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, st));
        RPY_CHECK(cudaStreamSynchronize(st));
        double dn = 0.0;
        for (int64_t i = 0; i < 3 * k; ++i) dn += (pr.got[i] - pr.ref[i]) * (pr.got[i] - pr.ref[i]);
        T.err = pr.rn > 0.0 ? std::sqrt(dn / pr.rn) : std::sqrt(dn);
        if (timed) {
            std::vector<float> ms;
            for (int q = 0; q < reps; ++q) {
                RPY_CHECK(cudaEventRecord(e0, st));
                r = rpy_forest_matvec(tree, f_dev, kT_over_eta_host, u, stream);
                if (r != RPY_OK) {
                    T.status = r;
                    return r;
                }
                RPY_CHECK(cudaEventRecord(e1, st));
                RPY_CHECK(cudaEventSynchronize(e1));
                float m = 0.f;
                RPY_CHECK(cudaEventElapsedTime(&m, e0, e1));
                ms.push_back(m);
            }
            std::sort(ms.begin(), ms.end());
            T.ms = ms[ms.size() / 2];
        }
        return RPY_OK;
    };
    auto record = [&](const Trial &T) {
        trials.push_back(T);
        if (out->n_trials < int(sizeof(out->trials) / sizeof(out->trials[0]))) {
            rpy_autotune_trial &o = out->trials[out->n_trials++];
            o.leaf_cap = T.prm.leaf_cap;
            o.order_p = T.prm.order_p;
            o.direct_w = T.prm.direct_w;
            o.direct_x = T.prm.direct_x;
            o.quad = T.prm.quad;
            o.est_rel_l2 = T.err;
            o.matvec_ms = T.ms;
            o.status = T.status;
        }
    };

    rpy_build_params base{};
    base.digits = digits;
    base.precision = precision;
    const int pdef = default_order(digits);
    int capdef = default_leaf_cap(digits);   // doubled below while its tree does not fit on the device
    const int plo = digits == 3 ? 4 : (digits == 6 ? 8 : 16), phi = digits == 3 ? 12 : (digits == 6 ? 24 : 27);
    base.leaf_cap = capdef;

    auto err_at = [&](int q, int p) -> Trial {
        rpy_build_params b = base;
        b.quad = q;
        b.order_p = p;
        Trial T;
        run(b, false, T, probe);
        record(T);
        return T;
    };
    // order for one quadrature rule: the smallest p whose sampled error meets
    // the goal, searched from p0; ok = false when no p does (the rule's own
    // error floor is above the goal), then p is the order of least error
    struct OrderPick {
        int p;
        double err;
        bool ok;
        int status;
    };
    auto search_p = [&](int q, int p0) -> OrderPick {
        int p = p0;
        Trial T0 = err_at(q, p);
        if (T0.status != RPY_OK) return {p, T0.err, false, T0.status};
        if (T0.err <= goal) {
            double e = T0.err;
            while (p - 1 >= plo) {
                Trial T = err_at(q, p - 1);
                if (T.status != RPY_OK) return {p, e, true, T.status};
                if (T.err > goal) break;
                --p;
                e = T.err;
            }
            return {p, e, true, RPY_OK};
        }
        double best_err = T0.err, prev = T0.err;
        int best_p = p;
        while (p + 1 <= phi) {
            ++p;
            Trial T = err_at(q, p);
            if (T.status == RPY_ERR_OOM) break;   // a higher order does not fit either
            if (T.status != RPY_OK) return {best_p, best_err, false, T.status};
            if (T.err < best_err) {
                best_err = T.err;
                best_p = p;
            }
            if (T.err <= goal) return {p, T.err, true, RPY_OK};
            if (T.err > 0.8 * prev) break;   // the rule's floor: a higher order no longer helps
            prev = T.err;
        }
        return {best_p, best_err, false, RPY_OK};
    };

    // quadrature rule and order: for a 6-digit target the cheaper rules are
    // tried as well; among the (rule, order) pairs that meet the goal the
    // fastest timed matvec wins
    std::vector<int> rules = digits == 3 ? std::vector<int>{3} : (digits == 6 ? std::vector<int>{6, 5, 4} : std::vector<int>{9});
    int best_q = rules[0], best_p = pdef;
    double best_ms = INFINITY, best_err = INFINITY;
    bool best_ok = false;
    int pstart = pdef;
    for (int q : rules) {
        OrderPick pk = search_p(q, pstart);
        // small leaf capacities on large uniform systems make millions of boxes, each
        // with its plane-wave expansions: double the capacity until the tree fits
        while (pk.status == RPY_ERR_OOM && capdef < 4096) {
            capdef *= 2;
            base.leaf_cap = capdef;
            pk = search_p(q, pstart);
        }
        RPY_TRY(pk.status);
        if (!pk.ok) {
            if (!best_ok && pk.err < best_err) {
                best_q = q;
                best_p = pk.p;
                best_err = pk.err;
            }
            continue;
        }
        rpy_build_params b = base;
        b.quad = q;
        b.order_p = pk.p;
        Trial T;
        int r = run(b, true, T, probe);
        record(T);
        RPY_TRY(r);
        if (T.err <= goal && (!best_ok || T.ms < best_ms)) {
            best_q = q;
            best_p = pk.p;
            best_ms = T.ms;
            best_err = T.err;
            best_ok = true;
        }
        pstart = pk.p;
    }
    base.quad = best_q;
    base.order_p = best_p;
    const int p = best_p;

    // leaf capacity, then the direct-substitution thresholds, by timed matvecs
    Trial best;
    bool have = false;
    auto consider = [&](const rpy_build_params &q) -> int {
        Trial T;
        int r = run(q, true, T, probe);
        record(T);
        if (r == RPY_ERR_OOM) return RPY_OK;   // a setting too large for the device is skipped
        RPY_TRY(r);
        bool ok = T.err <= goal;
        bool best_ok = have && best.err <= goal;
        if (!have || (ok && (!best_ok || T.ms < best.ms)) || (!ok && !best_ok && T.err < best.err)) {
            best = T;
            have = true;
        }
        return RPY_OK;
    };
    const double fcap[] = {0.5, 0.7, 1.0, 1.4, 2.0};
    for (double f : fcap) {
        rpy_build_params q = base;
        q.leaf_cap = std::max(8, int(std::lround(capdef * f)));
        RPY_TRY(consider(q));
    }
    if (!have) return RPY_ERR_INTERNAL;
    base = best.prm;
    const int dw = int(1.8 * ((p + 3) * (p + 4) / 2)), dx = int(0.6 * ((p + 1) * (p + 2) / 2));
    const int thr[][2] = {{-1, -1}, {dw / 2, dx / 2}, {2 * dw, 2 * dx}};
    for (const auto &w : thr) {
        rpy_build_params q = base;
        q.direct_w = w[0];
        q.direct_x = w[1];
        RPY_TRY(consider(q));
    }

    // verification on a fresh sample, four times the search's: half uniform over all
    // beads, half over the beads in the leaves of the chosen tree's two deepest levels
    // (the longest translation chains, and in the FP32 form the most rounding)
    const int64_t KV = std::min<int64_t>(4 * K, N);
    Probe vprobe;
    {
        std::vector<int64_t> deep;
        {
            rpy_tree tree = nullptr;
            RPY_TRY(rpy_forest_build(pos_dev, sys_offsets, nsys, a_host, &best.prm, stream, &tree));
            struct TreeGuard {
                rpy_tree t;
                ~TreeGuard() { rpy_tree_free(t); }
            } tgd{tree};
            auto fetch = [&](int field, std::vector<int> &v) -> int {
                int64_t bytes = 0;
                RPY_TRY(rpy_tree_export(tree, field, nullptr, 0, &bytes));
                v.resize(size_t(bytes) / sizeof(int));
                return rpy_tree_export(tree, field, v.data(), bytes, &bytes);
            };
            std::vector<int> perm, rng, lv, lvl;
            RPY_TRY(fetch(RPY_FIELD_PERM, perm));
            RPY_TRY(fetch(RPY_FIELD_BOX_RANGE, rng));
            RPY_TRY(fetch(RPY_FIELD_LEAVES, lv));
            RPY_TRY(fetch(RPY_FIELD_BOX_LEVEL, lvl));
            int top = 0;
            for (int b : lv) top = std::max(top, lvl[b]);
            for (int b : lv)
                if (lvl[b] >= top - 1)
                    for (int j = rng[2 * b]; j < rng[2 * b + 1]; ++j) deep.push_back(perm[j]);
        }
        uint64_t vseed = seed ^ 0xA5A5A5A5DEADBEEFull;
        std::set<int64_t> pick;
        const int64_t kd = std::min<int64_t>(KV / 2, int64_t(deep.size()));
        while (int64_t(pick.size()) < kd) pick.insert(deep[splitmix64(vseed) % uint64_t(deep.size())]);
        while (int64_t(pick.size()) < KV) pick.insert(int64_t(splitmix64(vseed) % uint64_t(N)));
        RPY_TRY(make_probe(std::vector<int64_t>(pick.begin(), pick.end()), vprobe));
    }
    const double vgoal = 0.5 * bound;
    Trial V;
    RPY_TRY(run(best.prm, false, V, vprobe));
    const int pmax = phi;
    for (int tries = 0; V.err > vgoal && tries < 4; ++tries) {
        rpy_build_params q = V.prm;
        if (q.precision == RPY_FP32) {
            // FP32 rounding or truncation?  The FP64 path at the same parameters decides
            rpy_build_params q64 = q;
            q64.precision = RPY_FP64;
            Trial V64;
            int r = run(q64, false, V64, vprobe);
            if (r == RPY_OK && V64.err <= vgoal) {
                V = V64;
                break;
            }
            if (r != RPY_OK && r != RPY_ERR_OOM) return r;
        }
        if (q.order_p + 1 > pmax) break;
        ++q.order_p;
        Trial Vn;
        int r = run(q, false, Vn, vprobe);
        if (r == RPY_ERR_OOM) break;
        RPY_TRY(r);
        V = Vn;
    }
    if (V.prm.order_p != best.prm.order_p || V.prm.precision != best.prm.precision) {
        // the verified choice differs from the search's: its own sampled error and time
        Trial T;
        RPY_TRY(run(V.prm, true, T, probe));
        record(T);
        best = T;
    }
    out->verify_rel_l2 = V.err;
    out->n_verify = int(KV);
    out->verify_ok = V.err <= vgoal ? 1 : 0;
    out->best = best.prm;
    out->est_rel_l2 = best.err;
    out->matvec_ms = best.ms;
    out->goal = goal;
    out->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return RPY_OK;
}
