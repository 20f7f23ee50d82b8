// Solid harmonics in the paper's normalisation (Sec. 2):
//   Y_n^m = sqrt((n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i m phi},  Y_n^{-m} = conj(Y_n^m),
// with the Condon-Shortley phase in P_n^m.  Regular y_n^m(v) = |v|^n Y_n^m,
// irregular z_n^m(v) = Y_n^m / |v|^{n+1}.  Only m >= 0 is stored (index tri(n, m)).
//
// Recurrences (Cartesian, no trigonometry):
//   y_0^0 = 1,  y_m^m = c_m (x + i y) y_{m-1}^{m-1},  c_m = -sqrt((2m-1)/(2m))
//   y_n^m = a_nm z y_{n-1}^m - b_nm r^2 y_{n-2}^m,
//           a_nm = (2n-1)/sqrt((n+m)(n-m)),  b_nm = sqrt((n+m-1)(n-m-1)/((n+m)(n-m)))
//   z_0^0 = 1/r, z_m^m = c_m (x + i y)/r^2 z_{m-1}^{m-1},
//   z_n^m = (a_nm z z_{n-1}^m - b_nm z_{n-2}^m) / r^2.
// Ladder relations of Sec. 2 restated for this normalisation (m >= 0):
//   d/dz y_n^m = sqrt((n+m)(n-m)) y_{n-1}^m,     (dx + i dy) y_n^m = sqrt((n-m-1)(n-m)) y_{n-1}^{m+1}
//   d/dz z_n^m = -sqrt((n+m+1)(n-m+1)) z_{n+1}^m, (dx + i dy) z_n^m = sqrt((n+m+2)(n+m+1)) z_{n+1}^{m+1}
#pragma once

#include "rpy_internal.h"

namespace rpy {

// Recurrence coefficients for degree <= p (host, double).
struct HarmRec {
    std::vector<double> a, b;   // [tri(n,m)]
    std::vector<double> c;      // [m]
};

inline HarmRec harm_rec(int p) {
    HarmRec h;
    int nc = ncoef(p + 2);
    h.a.assign(nc, 0.0);
    h.b.assign(nc, 0.0);
    h.c.assign(p + 3, 0.0);
    for (int m = 1; m <= p + 2; ++m) h.c[m] = -std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    for (int n = 1; n <= p + 2; ++n)
        for (int m = 0; m < n; ++m) {
            double nm = std::sqrt(double(n + m) * double(n - m));
            h.a[tri(n, m)] = (2.0 * n - 1.0) / nm;
            h.b[tri(n, m)] = std::sqrt(double(n + m - 1) * double(n - m - 1) > 0 ? double(n + m - 1) * double(n - m - 1) : 0.0) / nm;
        }
    return h;
}

// Generic recurrences with coefficient arrays (host or device memory).
template <typename T>
RPY_HD void regular_all(T x, T y, T z, int p, const T *ra, const T *rb, const T *rc, cpx<T> *out) {
    T r2 = x * x + y * y + z * z;
    cpx<T> diag = mk<T>(1, 0);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = rc[m] * (mk(x, y) * diag);
        out[tri(m, m)] = diag;
        cpx<T> prev2 = mk<T>(0, 0), prev1 = diag;
        for (int n = m + 1; n <= p; ++n) {
            int i = tri(n, m);
            cpx<T> cur = mk(ra[i] * z * prev1.x - rb[i] * r2 * prev2.x, ra[i] * z * prev1.y - rb[i] * r2 * prev2.y);
            out[i] = cur;
            prev2 = prev1;
            prev1 = cur;
        }
    }
}

template <typename T>
RPY_HD void irregular_all(T x, T y, T z, int p, const T *ra, const T *rb, const T *rc, cpx<T> *out) {
    T r2 = x * x + y * y + z * z;
    T ir2 = T(1) / r2;
    T ir = sqrt(ir2);
    cpx<T> diag = mk<T>(ir, 0);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = (rc[m] * ir2) * (mk(x, y) * diag);
        out[tri(m, m)] = diag;
        cpx<T> prev2 = mk<T>(0, 0), prev1 = diag;
        for (int n = m + 1; n <= p; ++n) {
            int i = tri(n, m);
            cpx<T> cur = mk((ra[i] * z * prev1.x - rb[i] * prev2.x) * ir2, (ra[i] * z * prev1.y - rb[i] * prev2.y) * ir2);
            out[i] = cur;
            prev2 = prev1;
            prev1 = cur;
        }
    }
}

}  // namespace rpy
