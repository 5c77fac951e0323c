// Contact tables for the matrix-free evaluation of f^E on the GPU.
//
// Sec. 2: f^E couples the stand's rail faces and the stock's contact faces
// through integrals over Gamma_R(t), the part of the rail covered by the
// stock at time t (M_B, C_B of Eq. defCB and b_X(t)). With faces that are
// axis-aligned rectangles in one plane, every (stand face, stock face)
// overlap is a rectangle. This file prepares, once per assembly:
//  - the interface DOFs (stand rail nodes, then stock contact nodes) and
//    each one's incident faces with the node's corner code;
//  - each face's rectangle (lo_u, lo_v, hi_u, hi_v) and its nodes by corner
//    code (bit 0: high u, bit 1: high v); stock faces in reference position;
//  - a uniform bin grid per body keyed by each face's low corner, with bins
//    at least as large as any face, so that all faces overlapping a query
//    rectangle lie in a small, fixed window of bins.
#include <algorithm>
#include <cmath>
#include <map>

#include "common.h"

namespace sdc {

namespace {

struct Rect {
    double lo_u, lo_v, hi_u, hi_v;
    int node_by_code[4];
};

// Classify one face; nodes are global DOF ids.
Rect face_rect(const std::vector<double>& xyz, const int64_t* q, int64_t dof_offset, int u, int v) {
    Rect r;
    double us[4], vs[4];
    for (int a = 0; a < 4; ++a) {
        us[a] = xyz[q[a] * 3 + u];
        vs[a] = xyz[q[a] * 3 + v];
    }
    r.lo_u = *std::min_element(us, us + 4);
    r.hi_u = *std::max_element(us, us + 4);
    r.lo_v = *std::min_element(vs, vs + 4);
    r.hi_v = *std::max_element(vs, vs + 4);
    const double eu = r.hi_u - r.lo_u, ev = r.hi_v - r.lo_v;
    if (!(eu > 0) || !(ev > 0)) throw ApiError(SDC_ERR_ARG, "degenerate contact face");
    int seen = 0;
    for (int a = 0; a < 4; ++a) {
        const bool hu = std::fabs(us[a] - r.hi_u) <= 1e-9 * eu;
        const bool lu = std::fabs(us[a] - r.lo_u) <= 1e-9 * eu;
        const bool hv = std::fabs(vs[a] - r.hi_v) <= 1e-9 * ev;
        const bool lv = std::fabs(vs[a] - r.lo_v) <= 1e-9 * ev;
        if (!(hu || lu) || !(hv || lv)) throw ApiError(SDC_ERR_ARG, "contact face is not an axis-aligned rectangle");
        const int code = (hu ? 1 : 0) | (hv ? 2 : 0);
        if (seen & (1 << code)) throw ApiError(SDC_ERR_ARG, "contact face is not an axis-aligned rectangle");
        seen |= 1 << code;
        r.node_by_code[code] = (int)(q[a] + dof_offset);
    }
    return r;
}

BinsHost make_bins(const std::vector<Rect>& R, size_t first, size_t count) {
    BinsHost b;
    if (count == 0) {
        b.nu = b.nv = 1;
        b.ptr.assign(2, 0);
        return b;
    }
    double ou = 1e300, ov = 1e300, mu = -1e300, mv = -1e300, bu = 0, bv = 0;
    for (size_t i = first; i < first + count; ++i) {
        ou = std::min(ou, R[i].lo_u);
        ov = std::min(ov, R[i].lo_v);
        mu = std::max(mu, R[i].lo_u);
        mv = std::max(mv, R[i].lo_v);
        bu = std::max(bu, R[i].hi_u - R[i].lo_u);
        bv = std::max(bv, R[i].hi_v - R[i].lo_v);
    }
    b.ou = ou;
    b.ov = ov;
    b.bu = bu * (1.0 + 1e-9);
    b.bv = bv * (1.0 + 1e-9);
    b.nu = (int)std::floor((mu - ou) / b.bu) + 1;
    b.nv = (int)std::floor((mv - ov) / b.bv) + 1;
    if ((int64_t)b.nu * b.nv > (1 << 26)) throw ApiError(SDC_ERR_ARG, "contact faces too uneven for binning");
    std::vector<int32_t> cnt((size_t)b.nu * b.nv + 1, 0);
    std::vector<int> bin_of(count);
    for (size_t i = 0; i < count; ++i) {
        const Rect& r = R[first + i];
        int iu = std::min(std::max((int)std::floor((r.lo_u - ou) / b.bu), 0), b.nu - 1);
        int iv = std::min(std::max((int)std::floor((r.lo_v - ov) / b.bv), 0), b.nv - 1);
        bin_of[i] = iv * b.nu + iu;
        cnt[bin_of[i] + 1]++;
    }
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    b.ptr = cnt;
    b.item.resize(count);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t i = 0; i < count; ++i) b.item[fill[bin_of[i]]++] = (int32_t)(first + i);
    return b;
}

}  // namespace

ContactHost build_contact(const BodyInput& stand, const BodyInput& stock, const std::vector<int64_t>& sq,
                          const std::vector<int64_t>& kq, const double dir[3]) {
    ContactHost C;
    const int64_t n_fix = stand.n_nodes(), n_mov = stock.n_nodes();
    const int64_t nsq = (int64_t)sq.size() / 4, nkq = (int64_t)kq.size() / 4;
    if (nsq == 0 || nkq == 0) throw ApiError(SDC_ERR_ARG, "empty contact face list");
    for (int64_t v : sq)
        if (v < 0 || v >= n_fix) throw ApiError(SDC_ERR_ARG, "stand contact node id out of range");
    for (int64_t v : kq)
        if (v < 0 || v >= n_mov) throw ApiError(SDC_ERR_ARG, "stock contact node id out of range");

    // common plane: the axis along which every contact node has the same coordinate
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v : sq)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], stand.xyz[v * 3 + i]);
            hi[i] = std::max(hi[i], stand.xyz[v * 3 + i]);
        }
    for (int64_t v : kq)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], stock.xyz[v * 3 + i]);
            hi[i] = std::max(hi[i], stock.xyz[v * 3 + i]);
        }
    double span = 0;
    for (int i = 0; i < 3; ++i) span = std::max(span, hi[i] - lo[i]);
    int normal = -1;
    for (int i = 0; i < 3; ++i)
        if (hi[i] - lo[i] <= 1e-12 * std::max(1.0, span)) normal = i;
    if (normal < 0) throw ApiError(SDC_ERR_ARG, "contact faces are not in one axis-aligned plane");
    if (std::fabs(dir[normal]) > 1e-12) throw ApiError(SDC_ERR_ARG, "motion direction leaves the contact plane");
    C.normal = normal;
    C.u = normal == 0 ? 1 : 0;
    C.v = normal == 2 ? 1 : 2;
    C.dir_u = dir[C.u];
    C.dir_v = dir[C.v];

    std::vector<Rect> R;
    R.reserve(nsq + nkq);
    for (int64_t f = 0; f < nsq; ++f) R.push_back(face_rect(stand.xyz, &sq[f * 4], 0, C.u, C.v));
    for (int64_t f = 0; f < nkq; ++f) R.push_back(face_rect(stock.xyz, &kq[f * 4], n_fix, C.u, C.v));
    C.nq_fix = (int)nsq;
    C.nq_mov = (int)nkq;

    // interface DOFs: sorted unique stand nodes, then stock nodes
    std::vector<int32_t> fixn, movn;
    for (int64_t v : sq) fixn.push_back((int32_t)v);
    for (int64_t v : kq) movn.push_back((int32_t)(v + n_fix));
    std::sort(fixn.begin(), fixn.end());
    fixn.erase(std::unique(fixn.begin(), fixn.end()), fixn.end());
    std::sort(movn.begin(), movn.end());
    movn.erase(std::unique(movn.begin(), movn.end()), movn.end());
    C.n_iface_fix = (int)fixn.size();
    C.dof = fixn;
    C.dof.insert(C.dof.end(), movn.begin(), movn.end());
    const int NI = (int)C.dof.size();
    C.pos.assign(n_fix + n_mov, -1);
    for (int a = 0; a < NI; ++a) C.pos[C.dof[a]] = a;

    // faces: rectangles and interface-local corner nodes
    C.rect.resize((size_t)4 * R.size());
    C.qnode.resize((size_t)4 * R.size());
    std::vector<std::vector<std::pair<int, int>>> inc(NI);
    for (size_t f = 0; f < R.size(); ++f) {
        C.rect[4 * f + 0] = R[f].lo_u;
        C.rect[4 * f + 1] = R[f].lo_v;
        C.rect[4 * f + 2] = R[f].hi_u;
        C.rect[4 * f + 3] = R[f].hi_v;
        for (int code = 0; code < 4; ++code) {
            const int a = C.pos[R[f].node_by_code[code]];
            C.qnode[4 * f + code] = a;
            inc[a].push_back({(int)f, code});
        }
    }
    C.inc_ptr.assign(NI + 1, 0);
    for (int a = 0; a < NI; ++a) {
        C.inc_ptr[a + 1] = C.inc_ptr[a] + (int)inc[a].size();
        for (auto& pr : inc[a]) {
            C.inc_quad.push_back(pr.first);
            C.inc_code.push_back(pr.second);
        }
    }
    C.bins_fix = make_bins(R, 0, nsq);
    C.bins_mov = make_bins(R, nsq, nkq);
    return C;
}

}  // namespace sdc
