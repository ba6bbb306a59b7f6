// Lattice Green's function of the 7-point Laplacian, FP64, for plan-time
// kernel tables (App. A, Eq. lgf3):
//
//   G(n) = - int_0^inf  Ie_{n1}(2t) Ie_{n2}(2t) Ie_{n3}(2t) dt,   Ie_k(x) = e^{-x} I_k(x).
//
// The half line is split at alpha (App. A): [0, alpha] by composite
// Gauss-Legendre on [0, 2^-6] and dyadic panels [2^e, 2^(e+1)]; [alpha, inf)
// analytically, from the product of the three large-argument expansions of I_k
// (Abramowitz & Stegun 9.7.1) integrated term by term.  alpha is a power of
// two >= max(2^10, 50 max|n_i|^2), where the expansion converges to 1e-17
// within a dozen terms.
//
// Ie_k(x) for all orders 0..K at one abscissa comes from Miller's backward
// recurrence I_{k-1} = (2k/x) I_k + I_{k+1}, normalised by the generating
// function identity Ie_0 + 2 sum_{k>=1} Ie_k = 1; for x >= 25 K^2 the
// asymptotic series is used directly.  The same Bessel row serves every
// triple, so a whole table costs one row per abscissa plus three products per
// (triple, abscissa).  Symmetry (Sec. 2.1): only sorted |n| triples are
// evaluated.
#include "lgf_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

namespace lgf {
namespace {

constexpr int kPanelNodes = 24;
constexpr int kFirstExp = -6;
constexpr int kAlphaMinExp = 10;
constexpr double kTailFactor = 50.0;
constexpr int kTailTerms = 12;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_q.
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // one more evaluation of the derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[q - 1 - i] = z;
        w[i] = w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// b_j with Ie_k(2t) ~ (4 pi t)^(-1/2) sum_j b_j t^(-j).
void expansion(int k, int nterms, double* b) {
    const double mu = 4.0 * k * k;
    double a = 1.0;
    b[0] = 1.0;
    for (int j = 1; j <= nterms; ++j) {
        a *= (mu - double(2 * j - 1) * double(2 * j - 1)) / (8.0 * j);
        b[j] = ((j & 1) ? -a : a) / std::ldexp(1.0, j);
    }
}

// Ie_k(x), k = 0..K, into out[0..K].
void scaled_bessel_row(double x, int K, double* out) {
    if (x == 0.0) {
        out[0] = 1.0;
        for (int k = 1; k <= K; ++k) out[k] = 0.0;
        return;
    }
    if (x >= 25.0 * double(K) * double(K) + 400.0) {
        const double pre = 1.0 / std::sqrt(2.0 * M_PI * x);
        for (int k = 0; k <= K; ++k) {
            const double mu = 4.0 * k * k;
            double term = 1.0, sum = 1.0;
            for (int j = 1; j < 60; ++j) {
                term *= -(mu - double(2 * j - 1) * double(2 * j - 1)) / (8.0 * j * x);
                sum += term;
                if (std::fabs(term) < 1e-18 * std::fabs(sum)) break;
            }
            out[k] = pre * sum;
        }
        return;
    }
    const int N = K + 40 + int(10.0 * std::sqrt(x));
    double ip1 = 0.0, ik = 1e-280, norm = 0.0;
    for (int k = 0; k <= K; ++k) out[k] = 0.0;
    for (int k = N; k >= 1; --k) {
        // ik holds I_k (scaled), ip1 holds I_{k+1}
        if (k <= K) out[k] = ik;
        norm += 2.0 * ik;
        const double im1 = (2.0 * k / x) * ik + ip1;
        ip1 = ik;
        ik = im1;
        if (ik > 1e250) {
            const double s = 1e-250;
            ik *= s;
            ip1 *= s;
            norm *= s;
            for (int j = k; j <= K && j <= N; ++j) out[j] *= s;
        }
    }
    out[0] = ik;
    norm += ik;
    const double inv = 1.0 / norm;
    for (int k = 0; k <= K; ++k) out[k] *= inv;
}

int alpha_exp(int cmax) {
    double need = std::max(std::ldexp(1.0, kAlphaMinExp), kTailFactor * double(cmax) * double(cmax));
    return int(std::ceil(std::log2(need)));
}

double tail(const int* k3, double alpha) {
    double b[3][kTailTerms + 1];
    for (int i = 0; i < 3; ++i) expansion(k3[i], kTailTerms, b[i]);
    double c[kTailTerms + 1];
    for (int J = 0; J <= kTailTerms; ++J) {
        double s = 0.0;
        for (int i = 0; i <= J; ++i)
            for (int j = 0; i + j <= J; ++j) s += b[0][i] * b[1][j] * b[2][J - i - j];
        c[J] = s;
    }
    double sum = 0.0;
    for (int J = kTailTerms; J >= 0; --J) sum += c[J] * std::pow(alpha, -0.5 - J) / (J + 0.5);
    return std::pow(4.0 * M_PI, -1.5) * sum;
}

}  // namespace

// G for sorted non-negative triples (a <= b <= c), FP64.
void green_sorted(const std::vector<std::array<int, 3>>& trip, std::vector<double>& out) {
    out.assign(trip.size(), 0.0);
    if (trip.empty()) return;
    int kmax = 0, emax = 0;
    for (auto& t : trip) kmax = std::max(kmax, t[2]);
    emax = alpha_exp(kmax);
    std::vector<double> gx, gw;
    gauss_legendre(kPanelNodes, gx, gw);
    std::vector<double> tq, wq;
    std::vector<double> edges{0.0};
    for (int e = kFirstExp; e <= emax; ++e) edges.push_back(std::ldexp(1.0, e));
    for (size_t p = 0; p + 1 < edges.size(); ++p) {
        const double a = edges[p], b = edges[p + 1];
        for (int i = 0; i < kPanelNodes; ++i) {
            tq.push_back(0.5 * (b - a) * gx[i] + 0.5 * (a + b));
            wq.push_back(0.5 * (b - a) * gw[i]);
        }
    }
    const int nq = int(tq.size());
    const int K = kmax;
    std::vector<double> bes(size_t(nq) * (K + 1));
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    {
        std::vector<std::thread> th;
        for (unsigned w = 0; w < nthr; ++w)
            th.emplace_back([&, w] {
                for (int q = int(w); q < nq; q += int(nthr))
                    scaled_bessel_row(2.0 * tq[q], K, &bes[size_t(q) * (K + 1)]);
            });
        for (auto& t : th) t.join();
    }
    std::vector<std::thread> th;
    const size_t n = trip.size();
    for (unsigned w = 0; w < nthr; ++w)
        th.emplace_back([&, w] {
            for (size_t i = w; i < n; i += nthr) {
                const auto& t = trip[i];
                const int ae = alpha_exp(t[2]);
                const int nuse = kPanelNodes * (1 + ae - kFirstExp);
                double s = 0.0;
                for (int q = 0; q < nuse; ++q) {
                    const double* r = &bes[size_t(q) * (K + 1)];
                    s += wq[q] * r[t[0]] * r[t[1]] * r[t[2]];
                }
                s += tail(t.data(), std::ldexp(1.0, ae));
                out[i] = -s;
            }
        });
    for (auto& t : th) t.join();
}

// Dense |offset| table T[(a*(V+1)+b)*(V+1)+c] = G(h*(a,b,c)), cached per (h, V).
std::shared_ptr<const std::vector<double>> green_abs_table(int h, int V) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::shared_ptr<const std::vector<double>>> cache;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find({h, V});
        if (it != cache.end()) return it->second;
    }
    std::vector<std::array<int, 3>> trip;
    for (int a = 0; a <= V; ++a)
        for (int b = a; b <= V; ++b)
            for (int c = b; c <= V; ++c) trip.push_back({h * a, h * b, h * c});
    std::vector<double> val;
    green_sorted(trip, val);
    const size_t W = size_t(V) + 1;
    auto tab = std::make_shared<std::vector<double>>(W * W * W);
    size_t idx = 0;
    for (int a = 0; a <= V; ++a)
        for (int b = a; b <= V; ++b)
            for (int c = b; c <= V; ++c, ++idx) {
                const double v = val[idx];
                const int p[3] = {a, b, c};
                static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                for (auto& pm : perm)
                    (*tab)[(size_t(p[pm[0]]) * W + p[pm[1]]) * W + p[pm[2]]] = v;
            }
    std::lock_guard<std::mutex> g(mu);
    cache[{h, V}] = tab;
    return tab;
}

}  // namespace lgf

extern "C" lgf_status lgf_green_values(const int32_t* n, int64_t count, double* out) {
    if (count < 0 || (count > 0 && (!n || !out)))
        return lgf::fail(LGF_ERR_INVALID_ARG, "lgf_green_values: bad arguments");
    std::vector<std::array<int, 3>> trip(static_cast<size_t>(count));
    for (int64_t i = 0; i < count; ++i) {
        int a[3] = {std::abs(n[3 * i]), std::abs(n[3 * i + 1]), std::abs(n[3 * i + 2])};
        std::sort(a, a + 3);
        if (a[2] > 4096) return lgf::fail(LGF_ERR_UNSUPPORTED, "lgf_green_values: |n_i| > 4096");
        trip[size_t(i)] = {a[0], a[1], a[2]};
    }
    std::vector<double> v;
    lgf::green_sorted(trip, v);
    std::memcpy(out, v.data(), sizeof(double) * size_t(count));
    return lgf::ok();
}
