// ritz.cpp -- the small eigenproblem of the deflated restart (host only).
//
// The deflated restart of Algorithm 1 (also used by Algorithm 2, whose Krylov operator is
// (tA)^{-1}) keeps k Ritz vectors of the projected matrix H_m (mp x mp, real, at most a few
// hundred rows): eigenpairs of H_m, the wanted ones (Algorithm 2: largest |mu|, Remark 4.1;
// Algorithm 1: smallest |theta|), complex eigenvectors split into their real and imaginary
// parts, orthonormalised into P_k.  The matrix is tiny, so it is solved on the host in
// FP64 with the textbook dense algorithm:
//   1. reduction to upper Hessenberg form by Householder reflections (accumulated in Q);
//   2. the Francis implicit double-shift QR iteration on the Hessenberg matrix, applied to
//      the whole matrix and accumulated in Q, until it is quasi upper triangular (the real
//      Schur form T = Q^T H Q, 1 x 1 blocks for real eigenvalues, 2 x 2 blocks for complex
//      pairs; a 2 x 2 block with real eigenvalues is split by one plane rotation);
//   3. eigenvectors of T by back substitution (real or complex), mapped back by Q;
//   4. selection and modified Gram-Schmidt (applied twice) for P_k.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <limits>
#include <vector>

#include "../../include/expm_block.h"

namespace {

using cd = std::complex<double>;

struct Mat {
    int n = 0;
    std::vector<double> a;   // column-major n x n
    explicit Mat(int n_ = 0) : n(n_), a((size_t)n_ * n_, 0.0) {}
    double& operator()(int r, int c) { return a[(size_t)c * n + r]; }
    double operator()(int r, int c) const { return a[(size_t)c * n + r]; }
};

// 1. Householder reduction to upper Hessenberg form: T <- Q^T T Q, Q accumulated.
void hessenberg(Mat& T, Mat& Q) {
    const int n = T.n;
    std::vector<double> v(n), w(n);
    for (int k = 0; k + 2 < n; ++k) {
        double xn = 0.0;
        for (int i = k + 1; i < n; ++i) xn = std::hypot(xn, T(i, k));
        if (xn == 0.0) continue;
        const double x0 = T(k + 1, k);
        const double alpha = x0 >= 0.0 ? -xn : xn;
        // v = x - alpha e_1, normalised (the reflector I - 2 v v^T maps x to alpha e_1)
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) {
            v[i] = T(i, k) - (i == k + 1 ? alpha : 0.0);
            vn = std::hypot(vn, v[i]);
        }
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; ++i) v[i] /= vn;
        // left: rows k+1.. of every column from k on
        for (int c = k; c < n; ++c) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += v[i] * T(i, c);
            for (int i = k + 1; i < n; ++i) T(i, c) -= 2.0 * s * v[i];
        }
        // right: columns k+1.. of every row
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += T(r, i) * v[i];
            for (int i = k + 1; i < n; ++i) T(r, i) -= 2.0 * s * v[i];
        }
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += Q(r, i) * v[i];
            for (int i = k + 1; i < n; ++i) Q(r, i) -= 2.0 * s * v[i];
        }
        T(k + 1, k) = alpha;
        for (int i = k + 2; i < n; ++i) T(i, k) = 0.0;
    }
}

// Apply the reflector I - 2 u u^T (u of length len, unit) to rows r0..r0+len-1 of T for
// columns c0..c1, and to columns r0.. of rows q0..q1 of T and of all rows of Q.
void reflect(Mat& T, Mat& Q, const double* u, int len, int r0, int c0, int c1, int q1) {
    for (int c = c0; c <= c1; ++c) {
        double s = 0.0;
        for (int i = 0; i < len; ++i) s += u[i] * T(r0 + i, c);
        for (int i = 0; i < len; ++i) T(r0 + i, c) -= 2.0 * s * u[i];
    }
    for (int r = 0; r <= q1; ++r) {
        double s = 0.0;
        for (int i = 0; i < len; ++i) s += T(r, r0 + i) * u[i];
        for (int i = 0; i < len; ++i) T(r, r0 + i) -= 2.0 * s * u[i];
    }
    for (int r = 0; r < Q.n; ++r) {
        double s = 0.0;
        for (int i = 0; i < len; ++i) s += Q(r, r0 + i) * u[i];
        for (int i = 0; i < len; ++i) Q(r, r0 + i) -= 2.0 * s * u[i];
    }
}

// Unit u with (I - 2 u u^T) x = beta e_1; false when x = 0.
bool householder(const double* x, int len, double* u) {
    double xn = 0.0;
    for (int i = 0; i < len; ++i) xn = std::hypot(xn, x[i]);
    if (xn == 0.0) return false;
    const double alpha = x[0] >= 0.0 ? -xn : xn;
    double un = 0.0;
    for (int i = 0; i < len; ++i) {
        u[i] = x[i] - (i == 0 ? alpha : 0.0);
        un = std::hypot(un, u[i]);
    }
    if (un == 0.0) return false;
    for (int i = 0; i < len; ++i) u[i] /= un;
    return true;
}

// Plane rotation [c s; -s c]^T on rows/columns (i, i+1), applied to all of T and Q.
void rotate(Mat& T, Mat& Q, int i, double c, double s) {
    const int n = T.n;
    for (int k = 0; k < n; ++k) {   // rows i, i+1:  G^T T
        const double a = T(i, k), b = T(i + 1, k);
        T(i, k) = c * a + s * b;
        T(i + 1, k) = -s * a + c * b;
    }
    for (int k = 0; k < n; ++k) {   // columns i, i+1:  T G
        const double a = T(k, i), b = T(k, i + 1);
        T(k, i) = c * a + s * b;
        T(k, i + 1) = -s * a + c * b;
    }
    for (int k = 0; k < n; ++k) {
        const double a = Q(k, i), b = Q(k, i + 1);
        Q(k, i) = c * a + s * b;
        Q(k, i + 1) = -s * a + c * b;
    }
}

// 2. Francis double-shift QR to the real Schur form.  Returns false if it does not converge.
bool schur(Mat& T, Mat& Q) {
    const int n = T.n;
    const double eps = std::numeric_limits<double>::epsilon();
    double anorm = 0.0;
    for (double x : T.a) anorm = std::max(anorm, std::fabs(x));
    if (anorm == 0.0) return true;
    int hi = n - 1, iter = 0, total = 0;
    while (hi >= 0) {
        // the active window [l, hi]: the largest l with a negligible subdiagonal at l
        int l = hi;
        for (; l > 0; --l) {
            double s = std::fabs(T(l - 1, l - 1)) + std::fabs(T(l, l));
            if (s == 0.0) s = anorm;
            if (std::fabs(T(l, l - 1)) <= eps * s) {
                T(l, l - 1) = 0.0;
                break;
            }
        }
        if (l == hi) {               // a 1 x 1 block has converged
            --hi;
            iter = 0;
            continue;
        }
        if (l == hi - 1) {           // a 2 x 2 block: split it when its eigenvalues are real
            const double a = T(hi - 1, hi - 1), b = T(hi - 1, hi), c = T(hi, hi - 1), d = T(hi, hi);
            const double p = 0.5 * (a - d), disc = p * p + b * c;
            if (disc >= 0.0) {
                // eigenvalue lam (the one farther from d), eigenvector (lam - d, c)
                const double lam = d + p + std::copysign(std::sqrt(disc), p);
                const double x = lam - d, y = c, r = std::hypot(x, y);
                if (r > 0.0) {
                    rotate(T, Q, hi - 1, x / r, y / r);
                    T(hi, hi - 1) = 0.0;
                }
            }
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++total > 100 * n) return false;
        ++iter;
        // shifts: the eigenvalues of the trailing 2 x 2 block, exceptional ones every 10
        double s, t;
        if (iter % 10 == 0) {
            const double e = std::fabs(T(hi, hi - 1)) + std::fabs(T(hi - 1, hi - 2));
            s = 1.5 * e;
            t = e * e;
        } else {
            s = T(hi - 1, hi - 1) + T(hi, hi);
            t = T(hi - 1, hi - 1) * T(hi, hi) - T(hi - 1, hi) * T(hi, hi - 1);
        }
        // first column of (T - s1 I)(T - s2 I) restricted to the window
        double x = T(l, l) * T(l, l) + T(l, l + 1) * T(l + 1, l) - s * T(l, l) + t;
        double y = T(l + 1, l) * (T(l, l) + T(l + 1, l + 1) - s);
        double z = T(l + 1, l) * T(l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            double v[3] = {x, y, z}, u[3];
            if (householder(v, 3, u)) {
                const int c0 = std::max(l, k - 1);
                reflect(T, Q, u, 3, k, c0, n - 1, std::min(k + 3, hi));
                if (k > l) {
                    T(k + 1, k - 1) = 0.0;
                    T(k + 2, k - 1) = 0.0;
                }
            }
            x = T(k + 1, k);
            y = T(k + 2, k);
            if (k < hi - 2) z = T(k + 3, k);
        }
        double v2[2] = {x, y}, u2[2];
        if (householder(v2, 2, u2)) {
            reflect(T, Q, u2, 2, hi - 1, hi - 2, n - 1, hi);
            T(hi, hi - 2) = 0.0;
        }
    }
    return true;
}

// 3. Eigenvectors of the quasi-triangular T by back substitution.  For the eigenvalue lam
// of block [k0, k1] (k1 = k0 for a real eigenvalue, k0 + 1 for a pair; lam with Im > 0),
// x solves (T - lam I) x = 0 with x_j = 0 beyond the block.
void schur_vector(const Mat& T, int k0, int k1, cd lam, double smin, std::vector<cd>& x) {
    const int n = T.n;
    x.assign(n, cd(0.0, 0.0));
    if (k0 == k1) {
        x[k0] = 1.0;
    } else {
        // the block [[a, b], [c, d]]: (a - lam) x0 + b x1 = 0  ->  x = (b, lam - a)
        x[k0] = T(k0, k1);
        x[k1] = lam - T(k0, k0);
    }
    for (int i = k0 - 1; i >= 0; --i) {
        const bool pair = i > 0 && T(i, i - 1) != 0.0;
        if (!pair) {
            cd r = 0.0;
            for (int j = i + 1; j <= k1; ++j) r += T(i, j) * x[j];
            cd den = T(i, i) - lam;
            if (std::abs(den) < smin) den = smin;
            x[i] = -r / den;
        } else {
            // rows i-1, i together: a 2 x 2 complex system
            cd r0 = 0.0, r1 = 0.0;
            for (int j = i + 1; j <= k1; ++j) {
                r0 += T(i - 1, j) * x[j];
                r1 += T(i, j) * x[j];
            }
            const cd a = T(i - 1, i - 1) - lam, b = T(i - 1, i), c = T(i, i - 1), d = T(i, i) - lam;
            cd det = a * d - b * c;
            if (std::abs(det) < smin * smin) det = smin * smin;
            x[i - 1] = (-r0 * d + b * r1) / det;
            x[i] = (-a * r1 + c * r0) / det;
            --i;
        }
        // keep the entries bounded (rescaling changes no direction)
        double mx = 0.0;
        for (int j = i; j <= k1; ++j) mx = std::max(mx, std::abs(x[j]));
        if (mx > 1e150)
            for (int j = 0; j <= k1; ++j) x[j] /= mx;
    }
}

struct Group {
    int k0, k1;      // Schur block
    cd lam;          // Im >= 0 for a pair
    double mod;
};

}  // namespace

namespace expm {

// Real Schur form and eigen-groups of an mp x mp matrix (column-major, ld).
bool ritz_groups(const double* H, int64_t ld, int n, Mat& T, Mat& Q, std::vector<Group>& g) {
    T = Mat(n);
    Q = Mat(n);
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r) {
            const double v = H[(size_t)c * ld + r];
            if (!std::isfinite(v)) return false;
            T(r, c) = v;
        }
    for (int i = 0; i < n; ++i) Q(i, i) = 1.0;
    hessenberg(T, Q);
    if (!schur(T, Q)) return false;
    g.clear();
    for (int k = 0; k < n;) {
        if (k + 1 < n && T(k + 1, k) != 0.0) {
            const double a = T(k, k), b = T(k, k + 1), c = T(k + 1, k), d = T(k + 1, k + 1);
            const double p = 0.5 * (a - d), disc = p * p + b * c;
            const cd lam(0.5 * (a + d), std::sqrt(std::max(0.0, -disc)));
            g.push_back({k, k + 1, lam, std::abs(lam)});
            k += 2;
        } else {
            g.push_back({k, k, cd(T(k, k), 0.0), std::fabs(T(k, k))});
            k += 1;
        }
    }
    return true;
}

}  // namespace expm

extern "C" expm_status expm_ritz_basis(const double* Hm, int64_t ldh, int mp, int k, int largest, int align,
                                       double* P, int64_t ldp, int* kept) {
    if (!Hm || !P || !kept || mp < 1 || ldh < mp || ldp < mp || k < 1 || k > mp || align < 1)
        return EXPM_INVALID_ARG;
    *kept = 0;
    Mat T, Q;
    std::vector<Group> g;
    if (!expm::ritz_groups(Hm, ldh, mp, T, Q, g)) return EXPM_NUMERICAL;
    // wanted order (stable: ties keep the Schur order)
    std::stable_sort(g.begin(), g.end(), [largest](const Group& a, const Group& b) {
        return largest ? a.mod > b.mod : a.mod < b.mod;
    });
    const int target = std::min(mp, (k + align - 1) / align * align);
    std::vector<Group> sel;
    int count = 0;
    for (const Group& x : g) {
        const int sz = x.k1 - x.k0 + 1;
        if (count + sz <= target) {
            sel.push_back(x);
            count += sz;
        }
        if (count == target) break;
    }
    while (count % align != 0 && !sel.empty()) {
        count -= sel.back().k1 - sel.back().k0 + 1;
        sel.pop_back();
    }
    if (count == 0) return EXPM_OK;
    // eigenvectors of H_m: y = Q x, split into real and imaginary parts
    double tn = 0.0;
    for (double x : T.a) tn = std::max(tn, std::fabs(x));
    const double smin = std::max(std::numeric_limits<double>::epsilon() * tn, std::numeric_limits<double>::min());
    std::vector<std::vector<double>> cols;
    std::vector<cd> x;
    for (const Group& s : sel) {
        schur_vector(T, s.k0, s.k1, s.lam, smin, x);
        std::vector<double> re(mp, 0.0), im(mp, 0.0);
        for (int r = 0; r < mp; ++r) {
            cd y = 0.0;
            for (int j = 0; j <= s.k1; ++j) y += Q(r, j) * x[j];
            re[r] = y.real();
            im[r] = y.imag();
        }
        cols.push_back(re);
        if (s.k1 > s.k0) cols.push_back(im);
    }
    // 4. orthonormalise: modified Gram-Schmidt, applied twice
    for (size_t c = 0; c < cols.size(); ++c) {
        std::vector<double>& v = cols[c];
        double n0 = 0.0;
        for (double e : v) n0 = std::hypot(n0, e);
        for (int pass = 0; pass < 2; ++pass)
            for (size_t q = 0; q < c; ++q) {
                double s = 0.0;
                for (int r = 0; r < mp; ++r) s += cols[q][r] * v[r];
                for (int r = 0; r < mp; ++r) v[r] -= s * cols[q][r];
            }
        double nv = 0.0;
        for (double e : v) nv = std::hypot(nv, e);
        if (!(nv > 1e-12 * n0) || !std::isfinite(nv)) return EXPM_NUMERICAL;   // dependent Ritz vectors
        for (double& e : v) e /= nv;
        for (int r = 0; r < mp; ++r) P[(size_t)c * ldp + r] = v[r];
    }
    *kept = count;
    return EXPM_OK;
}
