// Finite-element assembly of one body on the host (C++, OpenMP).
//
// Sec. 2, Eq. femContFix / femContMov and the matrices defined after
// Eq. femDiscr: with trilinear hexahedra,
//   K_ij    = int k grad phi_i . grad phi_j  +  int_{Gamma_env} h phi_i phi_j   (= -(A + B_env))
//   m_i     = int rho c phi_i                 (row-sum lumped mass)
//   genv_i  = int_{Gamma_env} h T_env phi_i   (= b_env)
// Volume integrals use 2x2x2 Gauss points on the isoparametric map, face
// integrals 2x2 points on the bilinear face; both are exact on boxes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>

#include "common.h"

namespace sdc {

namespace {

const int kCorner[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                           {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
const int kQuadCorner[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};

// Element stiffness (k-weighted) and lumped mass of one hexahedron.
// Returns false for a non-positive Jacobian.
bool hex_element(const double X[8][3], double k, double rho_c, double Ke[64], double me[8]) {
    const double g = 1.0 / std::sqrt(3.0);
    std::memset(Ke, 0, 64 * sizeof(double));
    std::memset(me, 0, 8 * sizeof(double));
    for (int gp = 0; gp < 8; ++gp) {
        const double xi[3] = {(gp & 1) ? g : -g, (gp & 2) ? g : -g, (gp & 4) ? g : -g};
        double N[8], dN[8][3];
        for (int a = 0; a < 8; ++a) {
            double f[3];
            for (int d = 0; d < 3; ++d) f[d] = 1.0 + kCorner[a][d] * xi[d];
            N[a] = 0.125 * f[0] * f[1] * f[2];
            dN[a][0] = 0.125 * kCorner[a][0] * f[1] * f[2];
            dN[a][1] = 0.125 * kCorner[a][1] * f[0] * f[2];
            dN[a][2] = 0.125 * kCorner[a][2] * f[0] * f[1];
        }
        // Jacobian J[i][d] = d x_i / d xi_d
        double J[3][3] = {{0}};
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                for (int d = 0; d < 3; ++d) J[i][d] += X[a][i] * dN[a][d];
        double cof[3][3];
        cof[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        cof[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        cof[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        cof[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        cof[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        cof[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * cof[0][0] + J[0][1] * cof[0][1] + J[0][2] * cof[0][2];
        if (!(det > 0.0)) return false;
        // grad phi_a = J^{-T} dN_a ; (J^{-1})[d][i] = cof[i][d] / det
        double G[8][3];
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                G[a][i] = (cof[i][0] * dN[a][0] + cof[i][1] * dN[a][1] + cof[i][2] * dN[a][2]) / det;
        const double wk = k * det, wm = rho_c * det;
        for (int a = 0; a < 8; ++a) {
            me[a] += wm * N[a];
            for (int b = 0; b < 8; ++b)
                Ke[a * 8 + b] += wk * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
        }
    }
    return true;
}

// int phi_a phi_b dS and int phi_a dS of one bilinear face.
void quad_face(const double X[4][3], double Fe[16], double fe[4]) {
    const double g = 1.0 / std::sqrt(3.0);
    std::memset(Fe, 0, 16 * sizeof(double));
    std::memset(fe, 0, 4 * sizeof(double));
    for (int gp = 0; gp < 4; ++gp) {
        const double xi[2] = {(gp & 1) ? g : -g, (gp & 2) ? g : -g};
        double N[4], t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
        for (int a = 0; a < 4; ++a) {
            const double f0 = 1.0 + kQuadCorner[a][0] * xi[0], f1 = 1.0 + kQuadCorner[a][1] * xi[1];
            N[a] = 0.25 * f0 * f1;
            const double d0 = 0.25 * kQuadCorner[a][0] * f1, d1 = 0.25 * kQuadCorner[a][1] * f0;
            for (int i = 0; i < 3; ++i) {
                t1[i] += X[a][i] * d0;
                t2[i] += X[a][i] * d1;
            }
        }
        const double cx = t1[1] * t2[2] - t1[2] * t2[1];
        const double cy = t1[2] * t2[0] - t1[0] * t2[2];
        const double cz = t1[0] * t2[1] - t1[1] * t2[0];
        const double dS = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int a = 0; a < 4; ++a) {
            fe[a] += dS * N[a];
            for (int b = 0; b < 4; ++b) Fe[a * 4 + b] += dS * N[a] * N[b];
        }
    }
}

int64_t find_col(const HostCSR& K, int64_t row, int64_t col) {
    const int32_t* b = K.col.data() + K.row_ptr[row];
    const int32_t* e = K.col.data() + K.row_ptr[row + 1];
    const int32_t* it = std::lower_bound(b, e, (int32_t)col);
    if (it == e || *it != col) return -1;
    return it - K.col.data();
}

}  // namespace

void assemble_body(const BodyInput& B, HostCSR& K, std::vector<double>& mass, std::vector<double>& genv) {
    const int64_t n = B.n_nodes(), ne = B.n_hex();
    if (n <= 0 || ne <= 0) throw ApiError(SDC_ERR_STATE, "body has no nodes or elements");
    if (n >= (int64_t)std::numeric_limits<int32_t>::max()) throw ApiError(SDC_ERR_ARG, "too many nodes");
    for (int64_t v : B.hex8)
        if (v < 0 || v >= n) throw ApiError(SDC_ERR_ARG, "hexahedron node id out of range");
    for (const auto& grp : B.robin)
        for (int64_t v : grp.quads)
            if (v < 0 || v >= n) throw ApiError(SDC_ERR_ARG, "Robin face node id out of range");

    // node -> element incidence
    std::vector<int64_t> inc_ptr(n + 1, 0), inc(ne * 8);
    for (int64_t v : B.hex8) inc_ptr[v + 1]++;
    for (int64_t i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
    {
        std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int a = 0; a < 8; ++a) inc[fill[B.hex8[e * 8 + a]]++] = e * 8 + a;
    }

    for (int64_t i = 0; i < n; ++i)
        if (inc_ptr[i + 1] - inc_ptr[i] > 64) throw ApiError(SDC_ERR_ARG, "node shared by more than 64 hexahedra");

    // element matrices
    std::vector<double> Ke((size_t)ne * 64), me((size_t)ne * 8);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t e = 0; e < ne; ++e) {
        double X[8][3];
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) X[a][i] = B.xyz[B.hex8[e * 8 + a] * 3 + i];
        const double k = B.k_hex.empty() ? B.k : B.k_hex[e];
        if (!hex_element(X, k, B.rho * B.c, &Ke[(size_t)e * 64], &me[(size_t)e * 8])) bad++;
    }
    if (bad) throw ApiError(SDC_ERR_ARG, "inverted or degenerate hexahedron");

    // sparsity pattern (sorted, unique neighbours)
    K.n = n;
    K.row_ptr.assign(n + 1, 0);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int32_t buf[512];
        int cnt = 0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1] && cnt + 8 <= 512; ++t) {
            const int64_t e = inc[t] / 8;
            for (int b = 0; b < 8; ++b) buf[cnt++] = (int32_t)B.hex8[e * 8 + b];
        }
        std::sort(buf, buf + cnt);
        K.row_ptr[i + 1] = std::unique(buf, buf + cnt) - buf;
    }
    for (int64_t i = 0; i < n; ++i) K.row_ptr[i + 1] += K.row_ptr[i];
    K.col.assign(K.row_ptr[n], 0);
    K.val.assign(K.row_ptr[n], 0.0);
    mass.assign(n, 0.0);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int32_t buf[512];
        int cnt = 0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1] && cnt + 8 <= 512; ++t) {
            const int64_t e = inc[t] / 8;
            for (int b = 0; b < 8; ++b) buf[cnt++] = (int32_t)B.hex8[e * 8 + b];
        }
        std::sort(buf, buf + cnt);
        const int u = (int)(std::unique(buf, buf + cnt) - buf);
        int32_t* cols = K.col.data() + K.row_ptr[i];
        double* vals = K.val.data() + K.row_ptr[i];
        std::copy(buf, buf + u, cols);
        double mi = 0.0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
            const int64_t e = inc[t] / 8;
            const int a = (int)(inc[t] % 8);
            mi += me[(size_t)e * 8 + a];
            for (int b = 0; b < 8; ++b) {
                const int32_t cb = (int32_t)B.hex8[e * 8 + b];
                const int pos = (int)(std::lower_bound(cols, cols + u, cb) - cols);
                vals[pos] += Ke[(size_t)e * 64 + a * 8 + b];
            }
        }
        mass[i] = mi;
    }

    // Robin faces, group by group: h int phi phi into K, h T_env int phi into genv
    genv.assign(n, 0.0);
    for (const auto& grp : B.robin) {
        if (grp.h == 0.0) continue;
        const int64_t nf = (int64_t)grp.quads.size() / 4;
        for (int64_t f = 0; f < nf; ++f) {
            double X[4][3], Fe[16], fe[4];
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) X[a][i] = B.xyz[grp.quads[f * 4 + a] * 3 + i];
            quad_face(X, Fe, fe);
            for (int a = 0; a < 4; ++a) {
                const int64_t ra = grp.quads[f * 4 + a];
                genv[ra] += grp.h * grp.T_env * fe[a];
                for (int b = 0; b < 4; ++b) {
                    const int64_t p = find_col(K, ra, grp.quads[f * 4 + b]);
                    if (p < 0) throw ApiError(SDC_ERR_ARG, "Robin face is not a face of a hexahedron");
                    K.val[p] += grp.h * Fe[a * 4 + b];
                }
            }
        }
    }
}

// The implied-column layout of K's FP32 copy (see ImpliedEll). Entries of a row run over its
// slice's table in increasing offset, that is in increasing column, as the CSR row does, so
// an SpMV that sums a row's entries in storage order adds the same products in the same order
// as the offsets form, with zeros between them. Slices are independent (OpenMP); the tables
// are deduplicated in slice order.
bool build_implied_ell(const HostCSR& K, ImpliedEll& out) {
    const int64_t n = K.n;
    if (n <= 0 || n >= (int64_t(1) << 30)) return false;
    int unsorted = 0;
#pragma omp parallel for schedule(static) reduction(| : unsorted)
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = K.row_ptr[r] + 1; k < K.row_ptr[r + 1]; ++k)
            if (K.col[k] <= K.col[k - 1]) unsorted = 1;
    if (unsorted) return false;
    const int64_t ns = (n + SLICE - 1) / SLICE;
    constexpr int W = IMPLIED_MAX_WIDTH;
    std::vector<int32_t> uni((size_t)ns * W);  // each slice's union, increasing
    std::vector<int32_t> width(ns, 0);
    std::vector<int64_t> wmax(ns, 0);          // longest row of the slice (offsets form)
    int too_wide = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : too_wide)
    for (int64_t s = 0; s < ns; ++s) {
        int32_t* u = uni.data() + (size_t)s * W;
        int w = 0;
        int32_t merged[2 * W];
        const int32_t* prev = nullptr;
        int64_t prev_len = -1;
        for (int64_t r = s * SLICE; r < std::min(n, (s + 1) * SLICE); ++r) {
            const int32_t* c = K.col.data() + K.row_ptr[r];
            const int64_t len = K.row_ptr[r + 1] - K.row_ptr[r];
            wmax[s] = std::max(wmax[s], len);
            // a row whose columns are its predecessor's shifted by one has the same offsets
            bool same = prev && len == prev_len;
            for (int64_t k = 0; same && k < len; ++k) same = c[k] == prev[k] + 1;
            prev = c;
            prev_len = len;
            if (same || too_wide) continue;
            // merge the row's offsets (increasing, since its columns are) into the union
            int a = 0, m = 0;
            int64_t k = 0;
            while ((a < w || k < len) && m <= W) {
                const int64_t o = k < len ? (int64_t)c[k] - r : INT64_MAX;
                if (a < w && (int64_t)u[a] < o) {
                    merged[m++] = u[a++];
                } else {
                    if (a < w && (int64_t)u[a] == o) ++a;
                    merged[m++] = (int32_t)o;
                    ++k;
                }
            }
            if (m > W) {
                too_wide = 1;
                continue;
            }
            std::copy(merged, merged + m, u);
            w = m;
        }
        width[s] = w;
    }
    if (too_wide) return false;
    out.slice_ptr.assign(ns + 1, 0);
    out.tab.assign(ns, 0);
    out.off.clear();
    std::map<std::vector<int32_t>, int32_t> seen;
    int64_t stored_offsets_form = 0;
    for (int64_t s = 0; s < ns; ++s) {
        const int32_t* u = uni.data() + (size_t)s * W;
        const int w = width[s];
        if (w == 0) return false;
        stored_offsets_form += wmax[s] * SLICE;
        // offsets increase, so the first row with the smallest and the last row with the
        // largest are the only ones that can leave [0, n)
        const int64_t r0 = s * SLICE, r1 = std::min(n, r0 + SLICE);
        const bool clamp = r0 + u[0] < 0 || (r1 - 1) + u[w - 1] >= n;
        std::vector<int32_t> key(u, u + w);
        int32_t t;
        const auto it = seen.find(key);
        if (it == seen.end()) {
            t = (int32_t)out.off.size();
            out.off.insert(out.off.end(), key.begin(), key.end());
            seen.emplace(std::move(key), t);
        } else {
            t = it->second;
        }
        out.tab[s] = clamp ? ~t : t;
        out.slice_ptr[s + 1] = out.slice_ptr[s] + (int64_t)w * SLICE;
    }
    if (out.slice_ptr[ns] * 4 > stored_offsets_form * 5) return false;
    out.val.assign(out.slice_ptr[ns], 0.0f);
    int missed = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : missed)
    for (int64_t s = 0; s < ns; ++s) {
        const int32_t* tab = out.off.data() + (out.tab[s] < 0 ? ~out.tab[s] : out.tab[s]);
        const int64_t w = (out.slice_ptr[s + 1] - out.slice_ptr[s]) / SLICE;
        for (int lane = 0; lane < SLICE; ++lane) {
            const int64_t r = s * SLICE + lane;
            if (r >= n) break;
            int64_t k = K.row_ptr[r];
            for (int64_t q = 0; q < w && k < K.row_ptr[r + 1]; ++q)
                if ((int64_t)K.col[k] - r == tab[q]) {
                    out.val[out.slice_ptr[s] + q * SLICE + lane] = (float)K.val[k];
                    ++k;
                }
            if (k != K.row_ptr[r + 1]) missed = 1;  // cannot happen: the table holds every offset
        }
    }
    return !missed;
}

}  // namespace sdc
