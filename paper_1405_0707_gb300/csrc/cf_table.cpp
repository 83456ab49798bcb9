// cf_table.cpp -- Caratheodory-Fejer (CF) poles and residues of e^x on (-inf, 0]
// (paper Section 2), computed on the host in double-double arithmetic.
//
// Construction (Section 2: SVD of the Hankel matrix of the Chebyshev coefficients of e^x
// transplanted from R^- to [-1, 1], partial-fraction form, eq. (11)):
//   1. x = s (w - 1)/(w + 1) maps w in [-1, 1] onto [-inf, 0]; F(w) = e^{x(w)}, s = 9.
//   2. Chebyshev coefficients c_0..c_K of F by the trapezoidal rule on the N + 1
//      Chebyshev-Lobatto points cos(pi j / N).
//   3. Hankel matrix H[i][j] = c_{i+j+1} (0 when i + j + 1 > K), K x K, real symmetric:
//      the eigenpair with the (nu+1)-st largest |eigenvalue| gives sigma and v.
//   4. The nu roots z of q(z) = sum_j v_j z^{K-1-j} outside the unit disk give the
//      poles tau = s (z - 1)^2 / (z + 1)^2.
//   5. Residues: least squares for omega_0 and the omega_i (conjugate pairs folded) on
//      M Chebyshev points of the first kind plus the point x = -inf.
// Parameters K = 100, N = 1024, M = 512.  Double-double (about 32 digits) makes the
// values, rounded to FP64, independent of the order of the arithmetic.
//
// Arithmetic: error-free transformations (Dekker 1971, Knuth's two-sum); products use
// std::fma for the exact rounding error.  Compile with -ffp-contract=off.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

namespace {

struct dd {
    double hi, lo;
};
inline dd mk(double a) { return {a, 0.0}; }
inline dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline dd fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline dd operator+(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline dd operator-(dd x) { return {-x.hi, -x.lo}; }
inline dd operator-(dd x, dd y) { return x + (-y); }
inline dd operator*(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p.hi, p.lo);
}
inline dd operator/(dd x, dd y) {
    double q1 = x.hi / y.hi;
    dd r = x - y * mk(q1);
    double q2 = r.hi / y.hi;
    r = r - y * mk(q2);
    double q3 = r.hi / y.hi;
    return fast_two_sum(q1, q2) + mk(q3);
}
inline bool operator<(dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
inline dd dabs(dd x) { return x.hi < 0 ? -x : x; }
inline dd dsqrt(dd x) {
    if (x.hi <= 0) return mk(0.0);
    double y = std::sqrt(x.hi);
    dd yy = mk(y);
    return yy + (x - yy * yy) * mk(0.5 / y);
}
inline dd dldexp(dd x, int e) { return {std::ldexp(x.hi, e), std::ldexp(x.lo, e)}; }

// atan(1/k) = sum_i (-1)^i / ((2i+1) k^(2i+1))
dd atan_inv(int k) {
    dd kk = mk((double)k), pw = mk(1.0) / kk, sum = mk(0.0), k2 = kk * kk;
    for (int i = 0; i < 60; ++i) {
        dd term = pw / mk((double)(2 * i + 1));
        sum = (i % 2 == 0) ? sum + term : sum - term;
        pw = pw / k2;
        if (std::fabs(pw.hi) < 1e-40) break;
    }
    return sum;
}
const dd& PI() {  // Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    static const dd v = mk(16.0) * atan_inv(5) - mk(4.0) * atan_inv(239);
    return v;
}
const dd& LN2() {  // ln 2 = 2 atanh(1/3) = 2 sum (1/3)^(2i+1)/(2i+1)
    static const dd v = [] {
        dd x = mk(1.0) / mk(3.0), pw = x, x2 = x * x, sum = mk(0.0);
        for (int i = 0; i < 80; ++i) {
            sum = sum + pw / mk((double)(2 * i + 1));
            pw = pw * x2;
        }
        return mk(2.0) * sum;
    }();
    return v;
}
dd dexp(dd x) {
    if (x.hi < -740.0) return mk(0.0);
    double k = std::nearbyint(x.hi / LN2().hi);
    dd r = x - LN2() * mk(k);
    r = dldexp(r, -10);
    dd term = mk(1.0), sum = mk(1.0);
    for (int i = 1; i <= 22; ++i) {
        term = term * r / mk((double)i);
        sum = sum + term;
    }
    for (int i = 0; i < 10; ++i) sum = sum * sum;
    return dldexp(sum, (int)k);
}
// Taylor series of cos / sin for |a| <= pi/4
dd dcos_small(dd a) {
    dd a2 = a * a, term = mk(1.0), sum = mk(1.0);
    for (int i = 1; i < 30; ++i) {
        term = -(term * a2 / mk((double)((2 * i - 1) * (2 * i))));
        sum = sum + term;
    }
    return sum;
}
dd dsin_small(dd a) {
    dd a2 = a * a, term = a, sum = a;
    for (int i = 1; i < 30; ++i) {
        term = -(term * a2 / mk((double)((2 * i) * (2 * i + 1))));
        sum = sum + term;
    }
    return sum;
}
// cos(pi m / N) for integer m, N divisible by 4
dd cospi_frac(long m, long N) {
    long mm = ((m % (2 * N)) + 2 * N) % (2 * N);
    if (mm > N) mm = 2 * N - mm;                  // cos is even, period 2N
    double sgn = 1.0;
    if (mm > N / 2) { mm = N - mm; sgn = -1.0; }  // cos(pi - a) = -cos a
    dd r;
    if (mm > N / 4) r = dsin_small(PI() * mk((double)(N / 2 - mm)) / mk((double)N));
    else r = dcos_small(PI() * mk((double)mm) / mk((double)N));
    return sgn < 0 ? -r : r;
}

struct cdd {
    dd re, im;
};
inline cdd operator+(cdd a, cdd b) { return {a.re + b.re, a.im + b.im}; }
inline cdd operator-(cdd a, cdd b) { return {a.re - b.re, a.im - b.im}; }
inline cdd operator*(cdd a, cdd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cdd operator/(cdd a, cdd b) {
    dd den = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
inline dd cabs2(cdd a) { return a.re * a.re + a.im * a.im; }

constexpr int K = 100, N = 1024, M = 512;
constexpr double S = 9.0;

struct Table {
    int nu = 0;
    std::vector<std::complex<double>> tau, omega;
    double omega0 = 0, sigma = 0;
    bool ok = false;
};

// Jacobi eigen-decomposition of a symmetric matrix in double (a starting point).
void jacobi_double(std::vector<double> A, int n, std::vector<double>& evals, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a(i, j) * a(i, j);
                if (i != j) off += a(i, j) * a(i, j);
            }
        if (off <= 1e-34 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a(p, q);
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    evals.resize(n);
    for (int i = 0; i < n; ++i) evals[i] = a(i, i);
}

// Solve (A) x = b in dd by Gaussian elimination with partial pivoting (A n x n row-major).
bool gauss_dd(std::vector<dd> A, std::vector<dd> b, int n, std::vector<dd>& x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (dabs(A[(size_t)piv * n + c]) < dabs(A[(size_t)r * n + c])) piv = r;
        if (A[(size_t)piv * n + c].hi == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            dd f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
            if (f.hi == 0.0) continue;
            for (int k = c; k < n; ++k) A[(size_t)r * n + k] = A[(size_t)r * n + k] - f * A[(size_t)c * n + k];
            b[r] = b[r] - f * b[c];
        }
    }
    x.assign(n, mk(0.0));
    for (int r = n - 1; r >= 0; --r) {
        dd acc = b[r];
        for (int k = r + 1; k < n; ++k) acc = acc - A[(size_t)r * n + k] * x[k];
        x[r] = acc / A[(size_t)r * n + r];
    }
    return true;
}

// Complex double arithmetic written out with the basic IEEE operations only (no libm, no
// libgcc complex division), so that the root finder takes the same path on every host.
struct cx {
    double re, im;
};
inline cx operator+(cx a, cx b) { return {a.re + b.re, a.im + b.im}; }
inline cx operator-(cx a, cx b) { return {a.re - b.re, a.im - b.im}; }
inline cx operator*(cx a, cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cx operator/(cx a, cx b) {   // Smith's algorithm
    if (std::fabs(b.re) >= std::fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.im + b.re * r;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
inline double cx_abs(cx a) { return std::sqrt(a.re * a.re + a.im * a.im); }

// All roots of sum_j v_j z^(deg-j), deg = v.size()-1, by the Aberth-Ehrlich iteration in
// complex double.  Starting points: a circle of radius 2^e with |v_deg / v_0| ~ 2^(e deg),
// at the angles pi m / Q (cos and sin from the double-double series above).
std::vector<cx> aberth(const std::vector<double>& v) {
    const int deg = (int)v.size() - 1;
    int e = 0;
    std::frexp(std::fabs(v[deg] / v[0]), &e);
    const double r0 = std::ldexp(1.0, e / deg);
    const long Q = 4000L * deg;                    // angle 2 pi (k + 1/4) / deg + 0.127 pi
    std::vector<cx> z(deg);
    for (int k = 0; k < deg; ++k) {
        const long m = 8000L * k + 2000L + 508L * deg;
        z[k] = {r0 * cospi_frac(m, Q).hi, r0 * cospi_frac(m - Q / 2, Q).hi};
    }
    const cx one{1.0, 0.0};
    for (int it = 0; it < 2000; ++it) {
        double maxrel = 0;
        for (int k = 0; k < deg; ++k) {
            cx p{v[0], 0.0}, dp{0.0, 0.0};
            for (int j = 1; j <= deg; ++j) {
                dp = dp * z[k] + p;
                p = p * z[k] + cx{v[j], 0.0};
            }
            cx ratio = p / dp, sum{0.0, 0.0};
            for (int j = 0; j < deg; ++j)
                if (j != k) sum = sum + one / (z[k] - z[j]);
            const cx w = ratio / (one - ratio * sum);
            z[k] = z[k] - w;
            maxrel = std::max(maxrel, cx_abs(w) / std::max(cx_abs(z[k]), 1e-300));
        }
        if (maxrel < 1e-15) break;
    }
    return z;
}

// Newton refinement of one root in complex dd.
cdd newton_dd(const std::vector<dd>& v, cx z0) {
    int deg = (int)v.size() - 1;
    cdd z{mk(z0.re), mk(z0.im)};
    for (int it = 0; it < 6; ++it) {
        cdd p{v[0], mk(0.0)}, dp{mk(0.0), mk(0.0)};
        for (int j = 1; j <= deg; ++j) {
            dp = dp * z + p;
            p = p * z + cdd{v[j], mk(0.0)};
        }
        z = z - p / dp;
    }
    return z;
}

Table build(int nu) {
    Table T;
    T.nu = nu;
    const dd s = mk(S);
    // step 2: F on the Lobatto points and the Chebyshev coefficients
    std::vector<dd> cosT(2 * N);
    for (int m = 0; m < 2 * N; ++m) cosT[m] = cospi_frac(m, N);
    std::vector<dd> F(N + 1);
    for (int j = 0; j <= N; ++j) {
        dd w = cosT[j];
        if (j == N) { F[j] = mk(0.0); continue; }
        F[j] = dexp(s * (w - mk(1.0)) / (w + mk(1.0)));
    }
    std::vector<dd> c(K + 1);
    for (int k = 0; k <= K; ++k) {
        dd acc = mk(0.0);
        for (int j = 0; j <= N; ++j) {
            dd term = F[j] * cosT[((long)j * k) % (2 * N)];
            if (j == 0 || j == N) term = term * mk(0.5);
            acc = acc + term;
        }
        c[k] = acc * mk(2.0) / mk((double)N);
    }
    c[0] = c[0] * mk(0.5);
    // step 3: Hankel eigenpair: double Jacobi, then inverse iteration in dd
    std::vector<dd> H((size_t)K * K, mk(0.0));
    std::vector<double> Hd((size_t)K * K, 0.0);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j)
            if (i + j + 1 <= K) { H[(size_t)i * K + j] = c[i + j + 1]; Hd[(size_t)i * K + j] = c[i + j + 1].hi; }
    std::vector<double> ev, V;
    jacobi_double(Hd, K, ev, V);
    std::vector<int> order(K);
    for (int i = 0; i < K; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(ev[a]) > std::fabs(ev[b]); });
    int want = order[nu];
    dd lam = mk(ev[want]);
    std::vector<dd> x(K);
    for (int i = 0; i < K; ++i) x[i] = mk(V[(size_t)i * K + want]);
    for (int it = 0; it < 4; ++it) {
        std::vector<dd> A = H;
        for (int i = 0; i < K; ++i) A[(size_t)i * K + i] = A[(size_t)i * K + i] - lam;
        std::vector<dd> y;
        if (!gauss_dd(A, x, K, y)) break;          // exact eigenvalue hit: keep x
        dd nrm = mk(0.0);
        for (int i = 0; i < K; ++i) nrm = nrm + y[i] * y[i];
        nrm = dsqrt(nrm);
        for (int i = 0; i < K; ++i) x[i] = y[i] / nrm;
        dd rq = mk(0.0);                            // Rayleigh quotient x^T H x
        for (int i = 0; i < K; ++i) {
            dd hx = mk(0.0);
            for (int j = 0; j < K; ++j) hx = hx + H[(size_t)i * K + j] * x[j];
            rq = rq + x[i] * hx;
        }
        lam = rq;
    }
    T.sigma = dabs(lam).hi;
    // step 4: roots outside the unit disk -> poles
    std::vector<double> vd(K);
    for (int i = 0; i < K; ++i) vd[i] = x[i].hi;
    auto roots = aberth(vd);
    std::vector<cdd> outside;
    for (auto& z : roots)
        if (cx_abs(z) > 1.0) outside.push_back(newton_dd(x, z));
    if ((int)outside.size() != nu) return T;
    std::vector<cdd> up;
    for (auto& z : outside) {
        cdd one{mk(1.0), mk(0.0)};
        cdd a = z - one, b = z + one;
        cdd t = cdd{s, mk(0.0)} * (a * a) / (b * b);
        if (t.im.hi > 0) up.push_back(t);
    }
    if ((int)up.size() != nu / 2) return T;
    std::sort(up.begin(), up.end(), [](const cdd& a, const cdd& b) { return b.im < a.im; });
    // step 5: least squares via Gram-Schmidt QR (twice) in dd
    int nc = 1 + 2 * (nu / 2), nr = M + 1;
    std::vector<std::vector<dd>> Acol(nc, std::vector<dd>(nr, mk(0.0)));
    std::vector<dd> rhs(nr, mk(0.0));
    for (int j = 0; j < M; ++j) {
        dd w = cosT[2 * j + 1];              // cos(pi (j + 1/2)/M), M = N/2
        dd xx = s * (w - mk(1.0)) / (w + mk(1.0));
        Acol[0][j] = mk(1.0);
        for (int i = 0; i < nu / 2; ++i) {
            cdd g = cdd{mk(1.0), mk(0.0)} / (cdd{xx, mk(0.0)} - up[i]);
            Acol[1 + 2 * i][j] = mk(2.0) * g.re;
            Acol[2 + 2 * i][j] = mk(-2.0) * g.im;
        }
        rhs[j] = dexp(xx);
    }
    Acol[0][M] = mk(1.0);                    // x = -inf: r = omega_0, e^x = 0
    std::vector<std::vector<dd>> R(nc, std::vector<dd>(nc, mk(0.0)));
    for (int k = 0; k < nc; ++k) {
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < k; ++i) {
                dd h = mk(0.0);
                for (int r = 0; r < nr; ++r) h = h + Acol[i][r] * Acol[k][r];
                for (int r = 0; r < nr; ++r) Acol[k][r] = Acol[k][r] - h * Acol[i][r];
                R[i][k] = R[i][k] + h;
            }
        dd nrm = mk(0.0);
        for (int r = 0; r < nr; ++r) nrm = nrm + Acol[k][r] * Acol[k][r];
        nrm = dsqrt(nrm);
        R[k][k] = nrm;
        for (int r = 0; r < nr; ++r) Acol[k][r] = Acol[k][r] / nrm;
    }
    std::vector<dd> qty(nc, mk(0.0)), sol(nc, mk(0.0));
    for (int k = 0; k < nc; ++k)
        for (int r = 0; r < nr; ++r) qty[k] = qty[k] + Acol[k][r] * rhs[r];
    for (int k = nc - 1; k >= 0; --k) {
        dd acc = qty[k];
        for (int i = k + 1; i < nc; ++i) acc = acc - R[k][i] * sol[i];
        sol[k] = acc / R[k][k];
    }
    T.omega0 = sol[0].hi;
    for (int i = 0; i < nu / 2; ++i) {
        T.tau.emplace_back(up[i].re.hi, up[i].im.hi);
        T.omega.emplace_back(sol[1 + 2 * i].hi, sol[2 + 2 * i].hi);
    }
    T.ok = true;
    return T;
}

std::mutex g_mu;
std::map<int, Table> g_cache;

}  // namespace

// Internal C++ entry used by the C ABI wrapper (api.cu).
bool expm_internal_cf_table(int nu, std::vector<std::complex<double>>& tau,
                            std::vector<std::complex<double>>& omega, double& omega0, double& sigma) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(nu);
    if (it == g_cache.end()) it = g_cache.emplace(nu, build(nu)).first;
    const Table& T = it->second;
    if (!T.ok) return false;
    tau = T.tau;
    omega = T.omega;
    omega0 = T.omega0;
    sigma = T.sigma;
    return true;
}
