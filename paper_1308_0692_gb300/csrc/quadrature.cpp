// Velocity sets of the library (host code): half-range and full-range Gauss-Hermite
// rules in double-double arithmetic, rounded to FP64.
//
// Table 1 of the paper lists the half-range rules D1Q^h_{2N}: the N Gauss nodes of
// the weight exp(-xi^2/2)/sqrt(2 pi) on [0, inf), mirrored to the negative half-line;
// the 2-D set is their tensor product.  This implementation follows Golub & Welsch's
// route through the moment matrix:
//   1. exact half-line moments m_k (Gamma function at half-integers);
//   2. Cholesky factor R of the Hankel matrix H_ij = m_{i+j}, H = R^T R, whose entries
//      give the Jacobi matrix: a_j = r_{j,j+1}/r_{jj} - r_{j-1,j}/r_{j-1,j-1},
//      b_j = r_{j+1,j+1}/r_{jj};
//   3. nodes = eigenvalues of the Jacobi matrix, isolated by Sturm-sequence bisection;
//   4. weights = 1 / sum_k p_k(x)^2 over the orthonormal polynomials (Christoffel).
// Full-range rules use the probabilists' Hermite recurrence a_j = 0, b_j = sqrt(j+1).
// Compiled with -ffp-contract=off: the error-free transformations below need every
// product and sum rounded separately.
#include <cmath>
#include <vector>

namespace lbmq {

struct dd {
    double hi, lo;
};

static inline dd two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

static inline dd quick_two_sum(double a, double b)
{
    double s = a + b;
    return {s, b - (s - a)};
}

static inline dd two_prod(double a, double b)
{
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}

static inline dd add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

static inline dd neg(dd a) { return {-a.hi, -a.lo}; }
static inline dd sub(dd a, dd b) { return add(a, neg(b)); }

static inline dd mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

static inline dd div(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = sub(a, mul(dd{q1, 0}, b));
    double q2 = r.hi / b.hi;
    r = sub(r, mul(dd{q2, 0}, b));
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return add(q, dd{q3, 0});
}

static inline dd sqrt_dd(dd a)
{
    if (a.hi <= 0) return {0, 0};
    double x = std::sqrt(a.hi);
    // one Newton step in double-double: x + (a - x^2) / (2x)
    dd xx{x, 0};
    dd r = sub(a, mul(xx, xx));
    dd corr = div(r, dd{2 * x, 0});
    dd y = add(xx, corr);
    r = sub(a, mul(y, y));
    corr = div(r, add(y, y));
    return add(y, corr);
}

static inline dd from(double v) { return {v, 0}; }
static inline bool less(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// pi in double-double (the two leading doubles of its binary expansion)
static const dd PI_DD = {3.141592653589793116e+00, 1.224646799147353207e-16};

// m_k = int_0^inf xi^k exp(-xi^2/2) dxi / sqrt(2 pi)
static std::vector<dd> halfline_moments(int count)
{
    dd inv_sqrt_2pi = div(from(1.0), sqrt_dd(mul(from(2.0), PI_DD)));
    std::vector<dd> m(count);
    for (int k = 0; k < count; ++k) {
        if (k % 2 == 0) {           // (k-1)!! / 2
            dd v = from(0.5);
            for (int j = 1; j < k; j += 2) v = mul(v, from(j));
            m[k] = v;
        } else {                    // 2^p p! / sqrt(2 pi), p = (k-1)/2
            dd v = inv_sqrt_2pi;
            int p = (k - 1) / 2;
            for (int j = 1; j <= p; ++j) v = mul(v, from(2.0 * j));
            m[k] = v;
        }
    }
    return m;
}

// Jacobi matrix (diagonal a[0..n-1], off-diagonal b[0..n-2]) and mu0 for n nodes.
static bool jacobi_halfline(int n, std::vector<dd> &a, std::vector<dd> &b, dd &mu0)
{
    int s = n + 1;
    std::vector<dd> mom = halfline_moments(2 * n + 1);
    std::vector<dd> R(s * s, from(0.0));
    for (int i = 0; i < s; ++i) {
        // R^T R = H, R upper triangular
        dd acc = mom[2 * i];
        for (int k = 0; k < i; ++k) acc = sub(acc, mul(R[k * s + i], R[k * s + i]));
        if (acc.hi <= 0) return false;
        dd rii = sqrt_dd(acc);
        R[i * s + i] = rii;
        for (int j = i + 1; j < s; ++j) {
            dd v = mom[i + j];
            for (int k = 0; k < i; ++k) v = sub(v, mul(R[k * s + i], R[k * s + j]));
            R[i * s + j] = div(v, rii);
        }
    }
    a.assign(n, from(0.0));
    b.assign(n > 1 ? n - 1 : 0, from(0.0));
    for (int j = 0; j < n; ++j) {
        dd t = div(R[j * s + j + 1], R[j * s + j]);
        if (j > 0) t = sub(t, div(R[(j - 1) * s + j], R[(j - 1) * s + j - 1]));
        a[j] = t;
        if (j + 1 < n) b[j] = div(R[(j + 1) * s + j + 1], R[j * s + j]);
    }
    mu0 = mom[0];
    return true;
}

static void jacobi_fullline(int n, std::vector<dd> &a, std::vector<dd> &b, dd &mu0)
{
    a.assign(n, from(0.0));
    b.assign(n > 1 ? n - 1 : 0, from(0.0));
    for (int j = 0; j + 1 < n; ++j) b[j] = sqrt_dd(from(j + 1.0));
    mu0 = from(1.0);
}

// number of eigenvalues of the Jacobi matrix below x (Sturm sequence of the LDL^T pivots)
static int count_below(const std::vector<dd> &a, const std::vector<dd> &b, dd x)
{
    int n = (int)a.size(), cnt = 0;
    dd q = sub(a[0], x);
    if (q.hi < 0) ++cnt;
    for (int k = 1; k < n; ++k) {
        if (q.hi == 0) q = from(1e-300);
        q = sub(sub(a[k], x), div(mul(b[k - 1], b[k - 1]), q));
        if (q.hi < 0) ++cnt;
    }
    return cnt;
}

// orthonormal polynomial values p_0..p_{n-1} at x (b_{k} p_{k+1} = (x - a_k) p_k - b_{k-1} p_{k-1})
static dd christoffel(const std::vector<dd> &a, const std::vector<dd> &b, dd mu0, dd x)
{
    int n = (int)a.size();
    dd pm1 = from(0.0);
    dd p = div(from(1.0), sqrt_dd(mu0));
    dd sum = mul(p, p);
    for (int k = 0; k + 1 < n; ++k) {
        dd t = mul(sub(x, a[k]), p);
        if (k > 0) t = sub(t, mul(b[k - 1], pm1));
        dd pn = div(t, b[k]);
        pm1 = p;
        p = pn;
        sum = add(sum, mul(p, p));
    }
    return div(from(1.0), sum);
}

// n-point Gauss rule from the Jacobi matrix; nodes ascending
static void gauss_from_jacobi(const std::vector<dd> &a, const std::vector<dd> &b, dd mu0,
                              std::vector<double> &x, std::vector<double> &w)
{
    int n = (int)a.size();
    // Gershgorin bound
    double lo = 0, hi = 0;
    for (int i = 0; i < n; ++i) {
        double r = 0;
        if (i > 0) r += std::fabs(b[i - 1].hi);
        if (i + 1 < n) r += std::fabs(b[i].hi);
        double l = a[i].hi - r - 1, h = a[i].hi + r + 1;
        if (i == 0 || l < lo) lo = l;
        if (i == 0 || h > hi) hi = h;
    }
    x.assign(n, 0);
    w.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        // k-th smallest eigenvalue: smallest t with count_below(t) >= k+1
        dd L = from(lo), H = from(hi);
        for (int it = 0; it < 200; ++it) {
            dd mid = mul(add(L, H), from(0.5));
            if (!less(L, mid) || !less(mid, H)) break;
            if (count_below(a, b, mid) >= k + 1) H = mid;
            else L = mid;
        }
        dd root = mul(add(L, H), from(0.5));
        x[k] = root.hi + root.lo;
        dd wk = christoffel(a, b, mu0, root);
        w[k] = wk.hi + wk.lo;
    }
}

}  // namespace lbmq

// 1-D rule of the library: nodes ascending, weights; returns false on failure.
bool lbm_rule_1d(int kind, int n, std::vector<double> &nodes, std::vector<double> &weights)
{
    using namespace lbmq;
    std::vector<dd> a, b;
    dd mu0;
    std::vector<double> x, w;
    if (kind == 0) {
        if (n < 1 || n > 8) return false;
        if (!jacobi_halfline(n, a, b, mu0)) return false;
        gauss_from_jacobi(a, b, mu0, x, w);
        nodes.clear();
        weights.clear();
        for (int i = n - 1; i >= 0; --i) {
            nodes.push_back(-x[i]);
            weights.push_back(w[i]);
        }
        for (int i = 0; i < n; ++i) {
            nodes.push_back(x[i]);
            weights.push_back(w[i]);
        }
        return true;
    }
    if (n < 2 || n > 16) return false;
    jacobi_fullline(n, a, b, mu0);
    gauss_from_jacobi(a, b, mu0, x, w);
    nodes.assign(n, 0);
    weights.assign(n, 0);
    for (int i = 0; i < n; ++i) {   // exact symmetry of the full-range rule
        nodes[i] = 0.5 * (x[i] - x[n - 1 - i]);
        weights[i] = 0.5 * (w[i] + w[n - 1 - i]);
    }
    if (n % 2 == 1) nodes[n / 2] = 0.0;
    return true;
}
