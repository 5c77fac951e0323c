// Host check of the implied-column layout of K's FP32 copy (build_implied_ell).
//
// Reads the two bodies' meshes (the binary written by tests/test_host_implied_ell.py),
// assembles K as the library does (assemble_body for each body, stand rows then stock rows),
// builds the stored-column sliced ELL (16-bit offsets from each slice's smallest column, or
// 32-bit columns when a slice spans more) and the implied-column layout, and runs the row loop
// of both GPU forms on the host: entries in storage order, CH entries a chunk, one fmaf chain
// per row. Checks that every index the implied form computes lies inside its array (values,
// tables, x) and that every row's FP32 sum is bitwise the stored-column form's, for two seeded
// vectors x and chunk widths 6 and 4. Prints one line: "implied <0|1> ..." and
// "bad <n> mismatches <n>"; exit status 0 when both counts are 0 (or the layout was refused).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "common.h"

using namespace sdc;

namespace {

bool read_body(FILE* f, BodyInput& b) {
    int64_t h[3];
    double m[3];
    if (fread(h, 8, 3, f) != 3 || fread(m, 8, 3, f) != 3) return false;
    b.set = true;
    b.k = m[0];
    b.rho = m[1];
    b.c = m[2];
    b.xyz.resize(h[0] * 3);
    b.hex8.resize(h[1] * 8);
    b.k_hex.resize(h[2]);
    return fread(b.xyz.data(), 8, b.xyz.size(), f) == b.xyz.size() &&
           fread(b.hex8.data(), 8, b.hex8.size(), f) == b.hex8.size() &&
           fread(b.k_hex.data(), 8, b.k_hex.size(), f) == b.k_hex.size();
}

struct Stored {
    std::vector<int64_t> sp;
    std::vector<int32_t> col;
    std::vector<float> val;
};

// the stored-column layout of build_ell: row entries in CSR order, padding (value 0, column of
// the row) at the end of each row
Stored stored_ell(const HostCSR& K) {
    const int64_t n = K.n, ns = (n + SLICE - 1) / SLICE;
    Stored S;
    S.sp.assign(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t r = s * SLICE; r < std::min(n, (s + 1) * SLICE); ++r)
            w = std::max(w, K.row_ptr[r + 1] - K.row_ptr[r]);
        S.sp[s + 1] = S.sp[s] + w * SLICE;
    }
    S.col.assign(S.sp[ns], 0);
    S.val.assign(S.sp[ns], 0.0f);
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t w = (S.sp[s + 1] - S.sp[s]) / SLICE;
        for (int lane = 0; lane < SLICE; ++lane) {
            const int64_t r = s * SLICE + lane;
            const int64_t len = r < n ? K.row_ptr[r + 1] - K.row_ptr[r] : 0;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t o = S.sp[s] + k * SLICE + lane;
                if (k < len) {
                    S.col[o] = K.col[K.row_ptr[r] + k];
                    S.val[o] = (float)K.val[K.row_ptr[r] + k];
                } else {
                    S.col[o] = (int32_t)std::min<int64_t>(r, n - 1);
                }
            }
        }
    }
    return S;
}

template <int CH>
float row_stored(const Stored& S, int64_t row, const std::vector<float>& x, long& bad) {
    const int64_t s = row >> 5, n = (int64_t)x.size();
    const int lane = (int)(row & 31);
    const int64_t b = S.sp[s], e = S.sp[s + 1];
    float acc = 0.0f;
    for (int64_t k0 = b + lane; k0 < e; k0 += (int64_t)CH * SLICE)
        for (int j = 0; j < CH; ++j) {
            const int64_t k = k0 + (int64_t)j * SLICE;
            const float v = k < e ? S.val[k] : 0.0f;
            const int64_t c = k < e ? S.col[k] : 0;
            if (c < 0 || c >= n) {
                ++bad;
                continue;
            }
            acc = std::fmaf(v, x[c], acc);
        }
    return acc;
}

// the row loop of the implied form (ell_row_implied): table position q advances by CH a chunk
template <int CH>
float row_implied(const ImpliedEll& ie, int64_t row, const std::vector<float>& x, long& bad) {
    const int64_t s = row >> 5, n = (int64_t)x.size();
    const int lane = (int)(row & 31);
    const int64_t b = ie.slice_ptr[s], e = ie.slice_ptr[s + 1];
    if ((e - b) % SLICE != 0 || ((e - b) * 4) % 16 != 0) ++bad;  // the bulk prefetch's size rule
    int32_t q = ie.tab[s];
    const bool clamp = q < 0;
    if (clamp) q = ~q;
    const int32_t r = (int32_t)row;
    float acc = 0.0f;
    for (int64_t k0 = b + lane; k0 < e; k0 += (int64_t)CH * SLICE, q += CH) {
        for (int j = 0; j < CH; ++j) {
            const int64_t k = k0 + (int64_t)j * SLICE;
            const bool in = k < e;
            if (in && (k >= (int64_t)ie.val.size() || q + j < 0 || q + j >= (int32_t)ie.off.size())) {
                ++bad;
                continue;
            }
            const float v = in ? ie.val[k] : 0.0f;
            int32_t c = in ? r + ie.off[q + j] : r;
            if (clamp) c = std::min(std::max(c, 0), (int32_t)n - 1);
            if (c < 0 || c >= n) {
                ++bad;
                continue;
            }
            acc = std::fmaf(v, x[c], acc);
        }
    }
    return acc;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    BodyInput b0, b1;
    const bool ok_read = read_body(f, b0) && read_body(f, b1);
    fclose(f);
    if (!ok_read) return 2;
    HostCSR K0, K1, K;
    std::vector<double> m0, m1, g0, g1;
    assemble_body(b0, K0, m0, g0);
    assemble_body(b1, K1, m1, g1);
    const int64_t nf = K0.n, nm = K1.n, n = nf + nm;
    K.n = n;
    K.row_ptr.assign(n + 1, 0);
    std::copy(K0.row_ptr.begin(), K0.row_ptr.end(), K.row_ptr.begin());
    for (int64_t i = 1; i <= nm; ++i) K.row_ptr[nf + i] = K0.row_ptr[nf] + K1.row_ptr[i];
    K.col = K0.col;
    for (int32_t c : K1.col) K.col.push_back(c + (int32_t)nf);
    K.val = K0.val;
    K.val.insert(K.val.end(), K1.val.begin(), K1.val.end());

    ImpliedEll ie;
    const bool ok = build_implied_ell(K, ie);
    printf("implied %d n %ld nnz %ld", ok ? 1 : 0, (long)n, (long)K.col.size());
    if (!ok) {
        printf("\n");
        return 0;
    }
    const Stored S = stored_ell(K);
    long clamp = 0;
    for (int32_t t : ie.tab) clamp += t < 0;
    printf(" stored %ld implied %ld tables %ld clamp_slices %ld\n", (long)S.sp.back(), (long)ie.slice_ptr.back(),
           (long)ie.off.size(), clamp);
    std::mt19937 g(7);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    long bad = 0, mism = 0;
    for (int trial = 0; trial < 2; ++trial) {
        std::vector<float> x(n);
        for (float& v : x) v = trial ? 1e-3f * nd(g) : 20.0f + nd(g);
        for (int64_t r = 0; r < n; ++r) {
            const float a6 = row_stored<6>(S, r, x, bad), a4 = row_stored<4>(S, r, x, bad);
            const float b6 = row_implied<6>(ie, r, x, bad), b4 = row_implied<4>(ie, r, x, bad);
            if (memcmp(&a6, &b6, 4) || memcmp(&a4, &b4, 4) || memcmp(&a6, &a4, 4)) ++mism;
        }
    }
    printf("bad %ld mismatches %ld\n", bad, mism);
    return (bad || mism) ? 1 : 0;
}
