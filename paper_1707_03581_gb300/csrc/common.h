// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <cstdint>
#include <limits>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sdcheat.h"

namespace sdc {

constexpr int SLICE = 32;       // rows per SELL slice (one warp)
constexpr int MAX_M = 16;       // standard nodes
constexpr int MAX_P = 64;       // embedded substeps per interval
constexpr int MAX_SOLVES = (SDC_MAX_SWEEPS + 1) * MAX_M;
constexpr int RED_BLOCK = 256;  // threads of the reduction kernels

// ----------------------------------------------------------------- host data

struct BodyInput {
    bool set = false;
    std::vector<double> xyz;      // n_nodes x 3
    std::vector<int64_t> hex8;    // n_hex x 8
    std::vector<double> k_hex;    // n_hex (empty = uniform)
    double k = 0, rho = 0, c = 0;
    struct RobinGroup {
        std::vector<int64_t> quads;  // n_faces x 4
        double h = 0, T_env = 0;
    };
    std::vector<RobinGroup> robin;   // Robin face groups (environment, cooling, floor ...)
    int64_t n_nodes() const { return (int64_t)xyz.size() / 3; }
    int64_t n_hex() const { return (int64_t)hex8.size() / 8; }
};

struct HostCSR {
    int64_t n = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
};

struct Weights {
    int kind = 0, M = 0, P = 0, w = 0;
    std::vector<double> c;      // M+1, c[0] = 0
    std::vector<double> emb;    // M x (P+1)
    std::vector<double> S;      // M x M
    std::vector<double> Shat;   // M x P
    std::vector<double> Stil;   // M x P x M
    std::vector<double> Semb;   // M x P x P
};

Weights make_weights(int kind, int M, int P, int window);
int window_start(int p, int P, int w);

// Assemble K = -(A + B_env) (CSR, sorted columns), lumped mass and b_env of one body.
void assemble_body(const BodyInput& b, HostCSR& K, std::vector<double>& mass, std::vector<double>& genv);

// FP32 copy of K with implied columns. Entry k of every row of slice s sits at
// slice_ptr[s] + 32 k + lane and belongs to column row + off[t_s + k], where the table
// off[t_s ..] is the increasing union of the relative columns (col - row) of the slice's
// rows; a row that lacks one of them holds 0 there. No column is stored: a 27-point stencil
// numbered plane by plane has a handful of distinct tables, shared by most slices.
// tab[s] = t_s, or ~t_s when some row of the slice would reach outside [0, n) with some
// offset of its table (the kernels clamp those columns; their entries are 0).
struct ImpliedEll {
    std::vector<int64_t> slice_ptr;  // n_slices + 1
    std::vector<int32_t> tab;        // n_slices
    std::vector<int32_t> off;        // the distinct tables, concatenated
    std::vector<float> val;          // slice_ptr[n_slices]
};
constexpr int IMPLIED_MAX_WIDTH = 64;  // entries a row of the implied layout at most

// Build the implied-column layout of K. Returns false (and leaves the other forms in use) when
// a row's columns are not increasing, n >= 2^30, a slice's union exceeds IMPLIED_MAX_WIDTH, or
// the layout stores more than 1.25 times the entries of the offsets form.
bool build_implied_ell(const HostCSR& K, ImpliedEll& out);

struct BinsHost {
    double ou = 0, ov = 0, bu = 1, bv = 1;
    int nu = 0, nv = 0;
    std::vector<int32_t> ptr, item;
};

// Contact tables built on the host (see ContactDev for the meaning).
struct ContactHost {
    int normal = 1, u = 0, v = 2;
    int n_iface_fix = 0;
    std::vector<int32_t> dof;
    std::vector<int32_t> inc_ptr, inc_quad, inc_code;
    std::vector<double> rect;      // 4 per quad
    std::vector<int32_t> qnode;    // 4 per quad, by corner code
    int nq_fix = 0, nq_mov = 0;
    BinsHost bins_fix, bins_mov;
    double dir_u = 0, dir_v = 0;
    std::vector<int32_t> pos;      // n_dof
};

ContactHost build_contact(const BodyInput& stand, const BodyInput& stock, const std::vector<int64_t>& stand_quads,
                          const std::vector<int64_t>& stock_quads, const double dir[3]);

// ----------------------------------------------------------------- device data

// Sliced ELL, slice height 32: entry (slice s, k, lane) at slice_ptr[s] + 32 k + lane.
// Column of an entry: base[s] + off[entry] when base[s] >= 0 (every column of the slice lies
// within 65,535 of the slice's smallest), else col[entry] (a wide slice; col is allocated only
// when the matrix has one). A 27-point stencil numbered plane by plane has slices spanning
// about two node planes, so its columns cost 2 bytes an entry instead of 4.
struct EllDev {
    int64_t n = 0;
    int64_t n_slices = 0;
    const int64_t* slice_ptr = nullptr;
    const int32_t* base = nullptr;
    const uint16_t* off = nullptr;
    const int32_t* col = nullptr;
    const double* val = nullptr;
    const float* val32 = nullptr;
    // Set when val32 holds the FP32 copy in the implied-column layout (ImpliedEll): its own
    // slice pointers, the per-slice table starts and the tables. NULL otherwise, and val32 is
    // then laid out like val.
    const int64_t* slice_ptr32 = nullptr;
    const int32_t* stab = nullptr;
    const int32_t* stoff = nullptr;
};

// Axis-aligned rectangle in the contact plane: x = lo_u, y = lo_v, z = hi_u, w = hi_v.
struct Rect4 {
    double x, y, z, w;
};

struct BinsDev {
    double ou = 0, ov = 0, bu = 1, bv = 1;   // origin and bin size
    double ibu = 1, ibv = 1;                // 1 / bin size
    int nu = 0, nv = 0;
    const int32_t* ptr = nullptr;           // nu*nv + 1
    const int32_t* item = nullptr;          // quad ids, stand quads or stock quads
};

// Contact tables. Interface DOFs: stand rail nodes first, then stock contact nodes.
struct ContactDev {
    int n_iface = 0;
    int n_iface_fix = 0;
    int nq_fix = 0, nq_mov = 0;            // quads: stand 0..nq_fix-1, stock nq_fix..
    const int32_t* dof = nullptr;          // n_iface global DOF ids
    const double* mass = nullptr;          // n_iface lumped masses
    const double* minv = nullptr;          // n_iface inverse lumped masses
    const double2* rinv = nullptr;         // per quad: 1 / (hi_u - lo_u), 1 / (hi_v - lo_v)
    const Rect4* dof_box = nullptr;        // per contact DOF: union of its faces (stock: reference position)
    Rect4 box_fix{}, box_mov{};            // union of each body's contact faces (stock: reference position)
    const int32_t* inc_ptr = nullptr;      // n_iface + 1
    const int32_t* inc_quad = nullptr;     // incident quad ids
    const int32_t* inc_code = nullptr;     // corner code of the node in that quad
    const Rect4* rect = nullptr;           // stock quads in reference position
    const int4* qnode = nullptr;           // interface-local node at corner codes 0..3
    BinsDev bins_fix, bins_mov;
    double dir_u = 0, dir_v = 0;           // in-plane components of the motion direction
    double z0 = 0, amp = 0, period = 0;
    double q0 = 0, h_c = 0;
    const int32_t* pos = nullptr;          // n_dof: interface-local index or -1
};

// Scalars of one CG solve (device).
// Scalars of one CG solve (device). Chronopoulos-Gear recurrences: gamma =
// (r, u), delta = (A u, u), rr = (r, r) of the current residual; alpha and
// gamma of the previous iteration are kept for the next step length.
struct CgState {
    double gamma, alpha, beta, bb, rr, delta;
    int iter;                  // updates applied
    int done;                  // stop flag (converged or capped)
    int runs;                  // executions of the SpMV kernel that did work
    int pending;               // FP32 loop: nx_* hold an update's step lengths not yet committed
    double nx_gamma, nx_alpha;
};

// Outer scalars of one mixed-precision solve (FP64 iterative refinement).
struct MixState {
    double bb, rr;             // ||b||^2 and ||b - A x||^2 (FP64)
    int passes;                // refinement passes done
    int done;
};

// Per-step device state.
struct StepState {
    double t0;                 // time origin
    double dt;
    long long n_done;          // macro steps completed since set_temperature
    int status;                // sticky sdc_status
    int loop_kernels;          // kernels run inside the CG/refinement loops of this step
    int cg_iters[MAX_SOLVES];
    int refinements[MAX_SOLVES];
    double residual[SDC_MAX_SWEEPS + 1];
    double heat[2];
    double friction_in;
    double rmax_partial_dummy;
    double true_res[MAX_SOLVES];  // ||b - A x|| / ||b|| with FP64 K after each mixed solve (if enabled)
};

// ----------------------------------------------------------------- helpers

#define SDC_CUDA_TRY(expr)                                                             \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) throw ::sdc::CudaError(_e, #expr, __FILE__, __LINE__);   \
    } while (0)

struct CudaError {
    cudaError_t code;
    std::string what;
    CudaError(cudaError_t c, const char* expr, const char* file, int line)
        : code(c),
          what(std::string(cudaGetErrorString(c)) + " in " + expr + " (" + file + ":" + std::to_string(line) + ")") {}
};

struct ApiError {
    sdc_status code;
    std::string what;
    ApiError(sdc_status c, std::string w) : code(c), what(std::move(w)) {}
};

}  // namespace sdc
