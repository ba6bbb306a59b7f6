// Choice of the interpolation stencil size n_max and the interval node count
// n_I = n_b + 1 for a target error (Sec. 2.5, the two-step procedure).
//
// Step 1 bounds the amplification of rounding errors: interpolating values
// perturbed by the working precision's unit roundoff eps_p perturbs the result
// by at most Lambda(X)^d eps_p (Eq. leb in d = 3 dimensions, tensor-product
// nodes), with Lambda the Lebesgue constant of the node set.  n_max is the
// largest node count n with Lambda_n^3 eps_p < eps, Lambda_n the Lebesgue
// constant of n equally spaced nodes: max over their interval of
// sum_i |l_i(x)|, l_i the Lagrange basis.
//
// Step 2 refines the intervals (more nodes, only the n_max nearest used)
// until the interpolation error of the function at hand is below eps.  The
// function the FLGF method interpolates is the field of well-separated
// sources: at a parent interval P' (nodes 2j, j = 0..n_b, spacing 2) the
// field of the nearest sources its interaction list can hold, on the face
// of the interval one interval width away (x = 4 n_b, y and z at the face's
// corners, edge midpoints and centre).  Each candidate n_b (the supported
// sizes 4..32, ascending, with n_I >= n_max) interpolates G(x - y) from P''s nodes to the
// nodes of its two children (spacing 1) with the Sec. 2.5 stencil, and the
// first whose maximum error relative to max |G| on the children's nodes is
// below eps is chosen.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "lgf_internal.h"

namespace lgf {
namespace {

// Lebesgue constant of n equispaced nodes 0..n-1: every sub-interval sampled,
// the best sample refined by golden-section search on its neighbourhood.
double lebesgue_equispaced(int n) {
    if (n <= 1) return 1.0;
    auto lam = [n](double x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            double l = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) l *= (x - j) / double(i - j);
            s += std::fabs(l);
        }
        return s;
    };
    constexpr int kSamples = 256;
    double best = 1.0, best_x = 0.0;
    for (int k = 0; k < n - 1; ++k)
        for (int q = 1; q < kSamples; ++q) {
            const double x = k + double(q) / kSamples;
            const double v = lam(x);
            if (v > best) {
                best = v;
                best_x = x;
            }
        }
    // golden-section refinement of the maximum within one sample step
    double a = std::max(0.0, best_x - 1.0 / kSamples), b = std::min(double(n - 1), best_x + 1.0 / kSamples);
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double c = b - g * (b - a), d = a + g * (b - a);
    double fc = lam(c), fd = lam(d);
    for (int it = 0; it < 80; ++it) {
        if (fc > fd) {
            b = d;
            d = c;
            fd = fc;
            c = b - g * (b - a);
            fc = lam(c);
        } else {
            a = c;
            c = d;
            fc = fd;
            d = a + g * (b - a);
            fd = lam(d);
        }
    }
    return std::max(best, std::max(fc, fd));
}

// Step-2 error of one (n_b, n_max): max over the source positions of the
// relative error of interpolating G(x - y) from the parent's nodes to its
// children's nodes.
double far_field_interp_error(int n_b, int n_max) {
    const int nI = n_b + 1, nc = 2 * n_b + 1;   // parent nodes, child nodes per axis
    const std::vector<double> W = interp_weights(n_b, n_max);
    // 1D matrix M[x][p]: weight of parent node p at child coordinate x = 0..2 n_b
    std::vector<double> M(size_t(nc) * nI, 0.0);
    for (int x = 0; x < nc; ++x) {
        const int c = x < n_b ? 0 : 1, i = x - c * n_b;
        for (int p = 0; p < nI; ++p) M[size_t(x) * nI + p] = W[(size_t(c) * nI + i) * nI + p];
    }
    // sources on the near face of the interval one parent width away
    std::vector<std::array<int, 3>> src;
    for (int a : {0, n_b, 2 * n_b})
        for (int b : {0, n_b, 2 * n_b}) src.push_back({4 * n_b, a, b});
    // every |offset| needed, evaluated once
    std::map<std::array<int, 3>, double> gval;
    auto key = [](int a, int b, int c) {
        std::array<int, 3> k{std::abs(a), std::abs(b), std::abs(c)};
        std::sort(k.begin(), k.end());
        return k;
    };
    for (const auto& y : src)
        for (int z = 0; z < nc; ++z)
            for (int yy = 0; yy < nc; ++yy)
                for (int x = 0; x < nc; ++x) gval[key(x - y[0], yy - y[1], z - y[2])] = 0.0;
    std::vector<std::array<int, 3>> trip;
    for (const auto& kv : gval) trip.push_back(kv.first);
    std::vector<double> val;
    green_sorted(trip, val);
    size_t idx = 0;
    for (auto& kv : gval) kv.second = val[idx++];
    auto G = [&](int a, int b, int c) { return gval.at(key(a, b, c)); };
    double worst = 0.0;
    std::vector<double> F(size_t(nI) * nI * nI), t1(size_t(nI) * nI * nc), t2(size_t(nI) * nc * nc);
    for (const auto& y : src) {
        // field at the parent's nodes (spacing 2), [pz][py][px]
        for (int pz = 0; pz < nI; ++pz)
            for (int py = 0; py < nI; ++py)
                for (int px = 0; px < nI; ++px)
                    F[(size_t(pz) * nI + py) * nI + px] = G(2 * px - y[0], 2 * py - y[1], 2 * pz - y[2]);
        // interpolate along x, then y, then z
        for (int pz = 0; pz < nI; ++pz)
            for (int py = 0; py < nI; ++py)
                for (int x = 0; x < nc; ++x) {
                    double s = 0.0;
                    for (int p = 0; p < nI; ++p) s += M[size_t(x) * nI + p] * F[(size_t(pz) * nI + py) * nI + p];
                    t1[(size_t(pz) * nI + py) * nc + x] = s;
                }
        for (int pz = 0; pz < nI; ++pz)
            for (int yy = 0; yy < nc; ++yy)
                for (int x = 0; x < nc; ++x) {
                    double s = 0.0;
                    for (int p = 0; p < nI; ++p) s += M[size_t(yy) * nI + p] * t1[(size_t(pz) * nI + p) * nc + x];
                    t2[(size_t(pz) * nc + yy) * nc + x] = s;
                }
        double emax = 0.0, gmax = 0.0;
        for (int z = 0; z < nc; ++z)
            for (int yy = 0; yy < nc; ++yy)
                for (int x = 0; x < nc; ++x) {
                    double s = 0.0;
                    for (int p = 0; p < nI; ++p) s += M[size_t(z) * nI + p] * t2[(size_t(p) * nc + yy) * nc + x];
                    const double g = G(x - y[0], yy - y[1], z - y[2]);
                    emax = std::max(emax, std::fabs(s - g));
                    gmax = std::max(gmax, std::fabs(g));
                }
        worst = std::max(worst, emax / gmax);
    }
    return worst;
}

}  // namespace
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status lgf_lebesgue_constant(int32_t n, double* out) {
    if (n < 1 || n > 40 || !out) return fail(LGF_ERR_INVALID_ARG, "lgf_lebesgue_constant: need 1 <= n <= 40 and out");
    *out = lebesgue_equispaced(n);
    return ok();
}

extern "C" lgf_status lgf_select_interp(double eps, int32_t precision, int32_t* n_max, int32_t* n_b,
                                        double* lebesgue, double* interp_err) {
    if (!(eps > 0.0 && eps < 1.0) || !n_max || !n_b || (precision != LGF_FP32 && precision != LGF_FP64))
        return fail(LGF_ERR_INVALID_ARG, "lgf_select_interp: need 0 < eps < 1, a precision and outputs");
    const double eps_p = precision == LGF_FP64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    // Step 1: the largest n with Lambda_n^3 eps_p < eps (at least 1 node)
    int nm = 1;
    double lam = 1.0;
    for (int n = 2; n <= 17; ++n) {
        const double l = lebesgue_equispaced(n);
        if (l * l * l * eps_p >= eps) break;
        nm = n;
        lam = l;
    }
    *n_max = nm;
    if (lebesgue) *lebesgue = lam;
    // Step 2: the smallest supported block size whose far-field interpolation
    // error is below eps
    double err = 0.0;
    int chosen = 0;
    for (int nb = 4; nb <= 32; nb += 2) {
        if (nb + 1 < nm) continue;
        err = far_field_interp_error(nb, nm);
        chosen = nb;
        if (err < eps) break;
    }
    *n_b = chosen;
    if (interp_err) *interp_err = err;
    if (chosen == 0 || err >= eps)
        return fail(LGF_ERR_UNSUPPORTED, "lgf_select_interp: no supported block size (4..32) reaches eps = " +
                                             std::to_string(eps) + " with n_max = " + std::to_string(nm) +
                                             " (largest tried: n_b = " + std::to_string(chosen) +
                                             ", error " + std::to_string(err) + ")");
    return ok();
}
