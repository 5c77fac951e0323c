// Quadrature nodes and MRSDC weight tables on the host, in long double.
//
// Sec. 3: standard nodes tau_m = t_n + dt c_m, embedded nodes
// tau_{m,p} = tau_{m-1} + p (tau_m - tau_{m-1}) / P, and the four tables
//   s_{m,j}      = int_{tau_{m-1}}^{tau_m}       l_j       (S)
//   shat_{m,q}   = sum_p s_{m,p,q}                         (Shat)
//   stil_{m,p,j} = int_{tau_{m,p-1}}^{tau_{m,p}} l_j       (Stil)
//   s_{m,p,q}    = int_{tau_{m,p-1}}^{tau_{m,p}} l^w_{m,q} (Semb)
// (Table 1). l_j are the Lagrange polynomials of the standard nodes and
// l^w_{m,q} those of a window of w consecutive embedded nodes around the
// substep (w = P reproduces the paper's definition; smaller w keeps the
// weights bounded for large P). shat is defined as the sum of the embedded
// weights so that the consistency identity stated after
// Eq. discrete-node-to-node-embedded holds by construction.
//
// Nodes are found by sign-change bracketing plus bisection on the Legendre
// recurrence; integrals use Gauss-Legendre rules exact for the polynomial
// degree, evaluating the Lagrange basis in product form.

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>
#include <utility>
#include <vector>

#include "common.h"

namespace sdc {

using ld = long double;

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
static void legendre(int n, ld x, ld* pn, ld* pn1) {
    ld p0 = 1.0L, p1 = x;
    if (n == 0) { *pn = 1.0L; *pn1 = 0.0L; return; }
    for (int k = 1; k < n; ++k) {
        ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

// All roots of f in (a, b) found by scanning for sign changes on a fine grid.
template <class F>
static std::vector<ld> roots_in(F f, ld a, ld b, int expected) {
    const int grid = 20000;
    std::vector<ld> out;
    ld xl = a, fl = f(a);
    for (int i = 1; i <= grid; ++i) {
        ld xr = a + (b - a) * i / grid;
        ld fr = f(xr);
        if (fl == 0.0L) {
            out.push_back(xl);
        } else if ((fl < 0) != (fr < 0) && fr != 0.0L) {
            ld lo = xl, hi = xr, flo = fl;
            for (int it = 0; it < 200; ++it) {
                ld mid = 0.5L * (lo + hi);
                ld fm = f(mid);
                if (fm == 0.0L) { lo = hi = mid; break; }
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
                if (hi - lo <= 4 * std::numeric_limits<ld>::epsilon()) break;
            }
            out.push_back(0.5L * (lo + hi));
        }
        xl = xr;
        fl = fr;
    }
    if ((int)out.size() != expected) throw std::runtime_error("node search failed");
    return out;
}

// Gauss-Legendre points/weights on [-1, 1].
static void gauss_legendre(int n, std::vector<ld>& x, std::vector<ld>& w) {
    auto f = [n](ld t) { ld a, b; legendre(n, t, &a, &b); return a; };
    x = roots_in(f, -1.0L, 1.0L, n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        ld pn, pn1;
        legendre(n, x[i], &pn, &pn1);
        // P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1)
        ld dp = n * (x[i] * pn - pn1) / (x[i] * x[i] - 1.0L);
        w[i] = 2.0L / ((1.0L - x[i] * x[i]) * dp * dp);
    }
}

std::vector<ld> standard_nodes_ld(int kind, int M) {
    std::vector<ld> c;
    if (kind == SDC_NODES_EQUI_NOLEFT) {
        for (int j = 1; j <= M; ++j) c.push_back((ld)j / M);
        return c;
    }
    if (kind == SDC_NODES_LOBATTO) {
        if (M < 2) throw std::runtime_error("Lobatto needs M >= 2");
        c.push_back(0.0L);
        if (M > 2) {
            int n = M - 1;  // interior points: zeros of P_n'
            auto dpn = [n](ld t) {
                ld pn, pn1;
                legendre(n, t, &pn, &pn1);
                return n * (pn1 - t * pn);  // (1 - t^2) P_n' up to sign, zero at interior roots
            };
            auto r = roots_in(dpn, -1.0L + 1e-12L, 1.0L - 1e-12L, M - 2);
            for (ld x : r) c.push_back(0.5L * (x + 1.0L));
        }
        c.push_back(1.0L);
        return c;
    }
    if (kind == SDC_NODES_RADAU_RIGHT) {
        // zeros of P_M - P_{M-1} on (-1, 1]; x = 1 is one of them
        auto f = [M](ld t) {
            ld pm, pm1;
            legendre(M, t, &pm, &pm1);
            return pm - pm1;
        };
        std::vector<ld> r;
        if (M > 1) r = roots_in(f, -1.0L + 1e-12L, 1.0L - 1e-9L, M - 1);
        for (ld x : r) c.push_back(0.5L * (x + 1.0L));
        c.push_back(1.0L);
        return c;
    }
    throw std::runtime_error("unknown node kind");
}

// int_a^b prod_{i != j} (s - x_i) / (x_j - x_i) ds, exactly for the degree.
static ld lagrange_integral(const std::vector<ld>& x, int j, ld a, ld b) {
    static std::mutex mu;
    static std::map<int, std::pair<std::vector<ld>, std::vector<ld>>> rules;
    const int deg = (int)x.size() - 1;
    const int ng = std::max(deg / 2 + 1, 1);
    std::vector<ld> gx, gw;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = rules.find(ng);
        if (it == rules.end()) {
            gauss_legendre(ng, gx, gw);
            rules[ng] = {gx, gw};
        } else {
            gx = it->second.first;
            gw = it->second.second;
        }
    }
    ld half = 0.5L * (b - a), mid = 0.5L * (a + b), acc = 0.0L;
    for (size_t g = 0; g < gx.size(); ++g) {
        ld s = mid + half * gx[g];
        ld v = 1.0L;
        for (size_t i = 0; i < x.size(); ++i)
            if ((int)i != j) v *= (s - x[i]) / (x[j] - x[i]);
        acc += gw[g] * v;
    }
    return acc * half;
}

int window_start(int p, int P, int w) { return std::min(std::max(p - w / 2, 1), P - w + 1); }

Weights make_weights(int kind, int M, int P, int window) {
    if (M < 1 || M > MAX_M) throw std::runtime_error("M out of range");
    if (P < 1 || P > MAX_P) throw std::runtime_error("P out of range");
    int w = window == 0 ? std::min(M, P) : window;
    if (w < 1 || w > P) throw std::runtime_error("window must be in [1, P]");
    std::vector<ld> std_nodes = standard_nodes_ld(kind, M);
    std::vector<ld> c(M + 1);
    c[0] = 0.0L;
    for (int m = 0; m < M; ++m) c[m + 1] = std_nodes[m];

    Weights W;
    W.kind = kind;
    W.M = M;
    W.P = P;
    W.w = w;
    W.c.resize(M + 1);
    W.emb.assign((size_t)M * (P + 1), 0.0);
    W.S.assign((size_t)M * M, 0.0);
    W.Shat.assign((size_t)M * P, 0.0);
    W.Stil.assign((size_t)M * P * M, 0.0);
    W.Semb.assign((size_t)M * P * P, 0.0);
    for (int m = 0; m <= M; ++m) W.c[m] = (double)c[m];
    std::vector<ld> shat((size_t)M * P, 0.0L);
    for (int m = 1; m <= M; ++m) {
        ld a = c[m - 1], b = c[m];
        std::vector<ld> e(P + 1);
        for (int p = 0; p <= P; ++p) {
            e[p] = p == 0 ? a : (p == P ? b : a + (b - a) * p / P);
            W.emb[(size_t)(m - 1) * (P + 1) + p] = (double)e[p];
        }
        if (a == b) continue;  // zero-length interval: every weight is zero
        for (int j = 0; j < M; ++j)
            W.S[(size_t)(m - 1) * M + j] = (double)lagrange_integral(std_nodes, j, a, b);
        for (int p = 1; p <= P; ++p) {
            for (int j = 0; j < M; ++j)
                W.Stil[((size_t)(m - 1) * P + (p - 1)) * M + j] =
                    (double)lagrange_integral(std_nodes, j, e[p - 1], e[p]);
            int j0 = window_start(p, P, w);
            std::vector<ld> win(e.begin() + j0, e.begin() + j0 + w);
            for (int qq = 0; qq < w; ++qq) {
                ld v = lagrange_integral(win, qq, e[p - 1], e[p]);
                W.Semb[((size_t)(m - 1) * P + (p - 1)) * P + (j0 - 1 + qq)] = (double)v;
                shat[(size_t)(m - 1) * P + (j0 - 1 + qq)] += v;
            }
        }
        for (int q = 0; q < P; ++q) W.Shat[(size_t)(m - 1) * P + q] = (double)shat[(size_t)(m - 1) * P + q];
    }
    return W;
}

}  // namespace sdc
