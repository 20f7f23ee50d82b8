// Algorithmic work of one matvec on a built tree, per stage: floating-point
// operations (an FMA counts 2) and DRAM bytes, the numerators of the roofline
// fractions that the benchmark reports beside the measured stage times.
//
// "Algorithmic" means the arithmetic and traffic the method needs at this
// tree, order p and plane-wave rule, counted from the tree itself (bead
// pairs of the near lists, boxes per level, present merge-and-shift sources
// per parent and direction, X-list and W-list sizes), not the instructions
// a kernel happens to issue:
//   P2P   per bead pair of the near lists (U lists and direct substitutes):
//         38 FLOP in FP64 (3 sub, r^2 5, Newton step of 1/sqrt 5, 1/r^2 1,
//         1/r^3 1, t1 2, 1 - 2a^2/r^2 2, c 1, R.F 5, t2 1, accumulate 12),
//         33 in FP32 (no Newton step: the reciprocal square root is a special-
//         function instruction); bytes: every bead's position and force read
//         once, its velocity written once.
//   P2M, P2L   per (bead, expansion): the regular or irregular solid harmonics
//         of degree p (10 FLOP per coefficient of the recurrence) and the four
//         charge sets accumulated into them (2 FMA per set and coefficient).
//   M2M, L2L   per child box: the per-octant translation of the four sets, as
//         the path computes it (rotation to the shift axis, m-diagonal z-shift,
//         rotation back; or, for the FP32 form below p = 12, the dense operator
//         restricted to its triangle); bytes: each expansion read and written
//         once per level pass.
//   M2X   per box: three frames x four sets x [A_k^m = sum_n c M (2 FMA per
//         coefficient and node) + the waves of a node from A (2 FMA per wave,
//         m and set, the two waves of angles a and pi - a sharing their
//         products)] plus the two frame rotations; bytes: M read, Xo written.
//   X2X   per (parent, direction): (present sources + children) x four sets
//         x S stored waves, one complex multiply-add (4 FMA) each; bytes: Xo
//         read once, Xi written once.
//   X2L   per box: the transpose of M2X; bytes: Xi read, L read and written.
//   EVAL  per bead of a leaf at level >= 2: harmonics of degree p and six
//         fields (2 FMA per coefficient each); per leaf the derived
//         expansions (18 x nc complex multiply-adds); per (bead, W-list box):
//         harmonics of degree p + 2 and 18 fields; bytes: L read, the derived
//         expansions written and read once per leaf, positions read and
//         velocities written.
// Polynomial far field (RPY_FLAG_CARTESIAN, N monomials of degree <= P): P2M per
// bead 2 multiplies and 4 FMA per monomial; M2M and L2L per child box and M2L per
// V-list pair one FMA per set and operator term (the pair counts of the tables);
// L2P per leaf the three velocity polynomials (about 10 FMA per coefficient) and
// per bead 3 FMA and 1 multiply per monomial; its M2L is timed under X2L.
#include <vector>

#include "rpy_internal.h"

namespace rpy {
namespace {

// FMAs of one factored rotation (z, y, z per degree) of one set; `quarter`: the
// frame rotations, whose y blocks are checkerboards (half the products).
double rot_fma(int p, bool quarter) {
    double f = 0;
    for (int n = 0; n <= p; ++n) {
        const double q = n + 1;
        f += 8 * q + (quarter ? 1.0 : 2.0) * q * q;
    }
    return f;
}

// FMAs of the m-diagonal z-shift of one set: output (n, m) takes the inputs of
// degrees m..n (M2M) or n..p (L2L), one real x complex product (2 FMA) each.
double zshift_fma(int p, bool up) {
    double f = 0;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) f += 2.0 * (up ? n - m + 1 : p - n + 1);
    return f;
}

// FMAs of the dense per-octant operator of one set (real layout, triangle only).
double dense_fma(int p, bool up) {
    const int nc = ncoef(p), D = 2 * nc;
    double f = 0;
    for (int r = 0; r < D; ++r) {
        int n = 0;
        while (tri(n + 1, 0) <= (r >> 1)) ++n;
        f += up ? 2.0 * ncoef(n) : double(D - 2 * tri(n, 0));
    }
    return f;
}

template <typename T>
int fetch(std::vector<T> &h, const T *d, size_t count) {
    h.resize(count);
    if (count == 0) return RPY_OK;
    RPY_CHECK(cudaMemcpy(h.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost));
    return RPY_OK;
}

}  // namespace
}  // namespace rpy

using namespace rpy;

extern "C" int rpy_tree_work(rpy_tree h, double *flops, double *bytes, int n) {
    Tree *tp = tree_of(h);
    if (!tp || !flops || !bytes || n < 0) return RPY_ERR_INVALID;
    Tree &t = *tp;
    if (!t.built) return RPY_ERR_STATE;
    DeviceGuard g(t.device);
    if (t.last_stream) RPY_CHECK(cudaStreamSynchronize(t.last_stream));
    double F[RPY_NUM_STAGES] = {}, B[RPY_NUM_STAGES] = {};
    const bool f32 = t.params.precision == RPY_FP32;
    const double w = f32 ? 4.0 : 8.0;                  // bytes of one real expansion value
    const int p = t.p, nc = ncoef(p), s = t.tabs->s, S = t.tabs->S;
    const double ce = 2 * w;                           // one complex value
    const int64_t N = t.n;

    // near field
    F[RPY_STAGE_P2P] = double(t.u_pairs + t.d_pairs) * (f32 ? 33.0 : 38.0);
    B[RPY_STAGE_P2P] = double(N) * (f32 ? (6 * 4 + 3 * 4 + 3 * 8) : (6 * 8 + 3 * 8));
    B[RPY_STAGE_GATHER] = double(N) * (3 * 8 + 4 + 3 * 8 + (f32 ? 3 * 4 : 0));   // forces, perm in; sorted out
    B[RPY_STAGE_COMBINE] = double(N) * (4 + 2 * 3 * 8 + 3 * 8);

    if (t.nlevels > 2 && (t.params.flags & RPY_FLAG_CARTESIAN)) {
        std::vector<int> lvl, beg, end, leaves;
        const size_t nb = size_t(t.nbox);
        RPY_TRY(fetch(lvl, t.b_level, nb));
        RPY_TRY(fetch(beg, t.b_begin, nb));
        RPY_TRY(fetch(end, t.b_end, nb));
        RPY_TRY(fetch(leaves, t.leaves, size_t(t.nleaf)));
        const int P = t.p, Nm = cart_terms(P);
        double pairs_l = 0, pairs_m = 0;   // M2L pairs (|a + b| <= P); M2M / L2L pairs (b <= a)
        for (int a0 = 0; a0 <= P; ++a0)
            for (int a1 = 0; a0 + a1 <= P; ++a1)
                for (int a2 = 0; a0 + a1 + a2 <= P; ++a2) {
                    pairs_l += cart_terms(P - a0 - a1 - a2);
                    pairs_m += double(a0 + 1) * (a1 + 1) * (a2 + 1);
                }
        double bead2 = 0, leaf2 = 0;
        for (int li = 0; li < t.nleaf; ++li) {
            const int b = leaves[li];
            if (lvl[b] < 2) continue;
            leaf2 += 1;
            bead2 += end[b] - beg[b];
        }
        const double n2 = double(nb - t.level_off[2]);
        const double nch = t.nlevels > 3 ? double(nb - t.level_off[3]) : 0.0;
        const double rw = w;   // real coefficients
        F[RPY_STAGE_P2M] = bead2 * Nm * (2 + 4 * 2);
        B[RPY_STAGE_P2M] = bead2 * 48 + leaf2 * 4 * Nm * rw;
        F[RPY_STAGE_M2M] = nch * pairs_m * 4 * 2;
        B[RPY_STAGE_M2M] = (nch + n2) * 4 * Nm * rw;
        F[RPY_STAGE_X2L] = double(t.n_v) * pairs_l * 4 * 2;
        B[RPY_STAGE_X2L] = n2 * 4 * Nm * rw * 2;   // every multipole read, every local written
        F[RPY_STAGE_L2L] = nch * pairs_m * 4 * 2;
        B[RPY_STAGE_L2L] = nch * 3 * 4 * Nm * rw;
        F[RPY_STAGE_EVAL] = leaf2 * 3 * Nm * 20.0 + bead2 * Nm * 7.0;
        B[RPY_STAGE_EVAL] = leaf2 * (4 + 2 * 3) * Nm * rw + bead2 * 48;
    } else if (t.nlevels > 2) {
        std::vector<int> lvl, beg, end, leaf, leaves, xoff, xidx, woff, coll, child, par;
        const size_t nb = size_t(t.nbox);
        RPY_TRY(fetch(lvl, t.b_level, nb));
        RPY_TRY(fetch(beg, t.b_begin, nb));
        RPY_TRY(fetch(end, t.b_end, nb));
        RPY_TRY(fetch(leaf, t.b_leaf, nb));
        RPY_TRY(fetch(leaves, t.leaves, size_t(t.nleaf)));
        RPY_TRY(fetch(xoff, t.x_off, nb + 1));
        RPY_TRY(fetch(xidx, t.x_idx, size_t(xoff[nb])));
        RPY_TRY(fetch(woff, t.w_off, size_t(t.nleaf) + 1));
        RPY_TRY(fetch(coll, t.b_coll, 27 * nb));
        RPY_TRY(fetch(child, t.b_child, 8 * nb));
        RPY_TRY(fetch(par, t.x2x_par, size_t(t.n_x2x_par)));
        const int b2 = t.level_off[2];
        const double n2 = double(nb - b2);
        const double nc2 = double(ncoef(p + 2));
        const double harm = 10.0 * nc, harm2 = 10.0 * nc2;
        // P2M: beads of leaves at level >= 2
        double bead2 = 0, leaf2 = 0, wpairs = 0;
        for (int li = 0; li < t.nleaf; ++li) {
            const int b = leaves[li];
            if (lvl[b] < 2) continue;
            leaf2 += 1;
            bead2 += end[b] - beg[b];
            wpairs += double(woff[li + 1] - woff[li]) * (end[b] - beg[b]);
        }
        F[RPY_STAGE_P2M] = bead2 * (harm + 4 * 2 * 2.0 * nc);
        B[RPY_STAGE_P2M] = bead2 * 48 + leaf2 * 4 * nc * ce;
        // P2L: (box, source bead) pairs of the X lists
        double xpairs = 0, xbox = 0;
        for (int b = b2; b < int(nb); ++b) {
            xbox += xoff[b + 1] > xoff[b] ? 1 : 0;
            for (int k = xoff[b]; k < xoff[b + 1]; ++k) xpairs += end[xidx[k]] - beg[xidx[k]];
        }
        F[RPY_STAGE_P2L] = xpairs * (harm + 4 * 2 * 2.0 * nc);
        B[RPY_STAGE_P2L] = xpairs * 48 + 2 * xbox * 4 * nc * ce;
        // M2M / L2L: child boxes at level >= 3
        const double nch = t.nlevels > 3 ? double(nb - t.level_off[3]) : 0.0;
        const bool rot = !f32 || p >= 12;
        const double m2m = rot ? 2 * rot_fma(p, false) + zshift_fma(p, true) : dense_fma(p, true);
        const double l2l = rot ? 2 * rot_fma(p, false) + zshift_fma(p, false) : dense_fma(p, false);
        F[RPY_STAGE_M2M] = nch * 4 * 2 * m2m;
        F[RPY_STAGE_L2L] = nch * 4 * 2 * l2l;
        double npar = 0;
        for (int b = b2; b < int(nb); ++b) npar += leaf[b] ? 0 : 1;
        B[RPY_STAGE_M2M] = (nch + npar) * 4 * nc * ce;
        B[RPY_STAGE_L2L] = (nch * 2 + npar) * 4 * nc * ce;
        // plane waves
        const double conv = 3 * 4 * (2.0 * nc * s + 2.0 * S * (p + 1)) + 2 * 4 * rot_fma(p, true);
        F[RPY_STAGE_M2X] = n2 * 2 * conv;
        F[RPY_STAGE_X2L] = n2 * 2 * conv;
        B[RPY_STAGE_M2X] = n2 * (4 * nc + 6.0 * 4 * S) * ce;
        B[RPY_STAGE_X2L] = n2 * (6.0 * 4 * S + 2 * 4 * nc) * ce;
        double units = 0;
        const OpTables &tb = *t.tabs;
        for (int P : par)
            for (int d = 0; d < kDirs; ++d) {
                const int ng = tb.grp_n[d];
                const int nsl = tb.grp_off[d * (kGroupMax + 1) + ng];
                for (int z = 0; z < nsl; ++z) {
                    const int sl = tb.slot_list[d * 216 + z] & 255, q = sl >> 3, o = sl & 7;
                    const int Q = coll[27 * size_t(P) + q];
                    if (Q >= 0 && !leaf[Q] && child[8 * size_t(Q) + o] >= 0) units += 1;
                }
                for (int c = 0; c < 8; ++c) units += child[8 * size_t(P) + c] >= 0 ? 1 : 0;
            }
        F[RPY_STAGE_X2X] = units * 4 * S * 4 * 2.0;
        B[RPY_STAGE_X2X] = 2 * n2 * 6.0 * 4 * S * ce;
        // L2P with Eq. (2.8) at the beads, the derived expansions per leaf, M2P of large W boxes
        F[RPY_STAGE_EVAL] = bead2 * (harm + 6 * 2 * 2.0 * nc) + leaf2 * 18 * nc * 8.0 +
                            wpairs * (harm2 + 18 * 2 * 2.0 * nc2);
        B[RPY_STAGE_EVAL] = leaf2 * (4 * nc + 2 * 18 * nc) * ce + bead2 * 48;
    }
    for (int k = 0; k < n; ++k) {
        flops[k] = k < RPY_NUM_STAGES ? F[k] : 0.0;
        bytes[k] = k < RPY_NUM_STAGES ? B[k] : 0.0;
    }
    return RPY_OK;
}
