// Kernel argument blocks and launch entry points (device side of the stepper).
#pragma once

#include "common.h"

namespace sdc {

constexpr int MAXE = 32;            // coupling entries per contact DOF and substep time
constexpr int GEOM_THREADS = 64;    // threads per block of k_iface_geom (one slot per block row)
constexpr int IFACE_MAX_CLUSTER = 16;   // CTAs of the substep-loop cluster (at most)
constexpr int IFACE_TARGET_CHUNK = 128;  // preferred contact DOFs per CTA of the loop
constexpr int IFACE_THREADS = 512;      // threads per CTA of that cluster
constexpr int IFACE_PER_THREAD = 2;     // contact DOFs one thread of a shared-memory-replica loop owns
constexpr int IFACE_PER_THREAD_GL = 4;  // the same for the global-replica loop
constexpr int IFACE_BATCH = 8;          // coupling entries fetched per round
// largest contact interface the loop takes (global replicas, 16 CTAs x 512 threads x 4)
constexpr int IFACE_MAX_NI = 32768;

enum RhsMode { RHS_GIVEN = 0, RHS_PRED = 1, RHS_SWEEP = 2 };

// One Jacobi-PCG solve of (diag(m) + dtau K) x = b in the Chronopoulos-Gear
// arrangement: per iteration one kernel forms w = A u and the three dot
// products (one global reduction), a second updates the vectors.
// Precomputed coupling operator f^E(T, tau_s)_a = cst[s][a] + sum_k coef[s][k][a] T_I[idx[s][k][a]].
struct CouplingOp {
    int32_t* cnt;     // [slots][NI]
    int32_t* idx;     // [slots][MAXE][NI]
    double* coef;     // [slots][MAXE][NI]
    double* cst;      // [slots][NI]
    float* coef32;    // [slots][MAXE][NI] FP32 copy (mixed precision), or NULL
};

// The contact coupling in the matrix of fully implicit Euler (see ie_contact).
struct IeOp {
    const int32_t* pos;             // DOF -> contact index or -1
    const int32_t* dof;             // contact index -> DOF
    CouplingOp E;                   // the step's coupling rows; indices are contact-DOF ids
    int slot, NI;
};

struct CgArgs {
    EllDev A;
    const double* mass;
    const double* diagK;
    double dtau;
    int64_t n;
    double *X, *R, *U, *P, *W, *S, *D;  // iterate, residual, u = D r, direction, A u, A p, 1/diag
    CgState* cg;
    int* loop_kernels;              // StepState::loop_kernels
    double* partials;
    double* gpartials;              // group totals of the two-level reduction
    unsigned int* counter;          // [0] groups done, [1 + g] blocks of group g done
    int* iters_out;                 // iteration count of this solve
    int* status;                    // sticky status word
    int max_iter;
    int tail_pairs;                 // (spmv, update) pairs after this one in the graph's loop body
    double rtol2;
    unsigned long long handle;      // cudaGraphConditionalHandle of the enclosing while node
    IeOp ie;                        // k_ie_init / k_ie_spmv only
};

// One mixed-precision solve of (diag(m) + dtau K) x = b: FP64 residuals
// r = b - A x around FP32 Jacobi-PCG solves of A d = r (iterative refinement).
// Largest grid of the FP32 SpMV whose dot partials every block of the update
// sums itself (above it: last-block reduction in the SpMV).
constexpr int MIX_DEFER_MAX_BLOCKS = 2048;
constexpr int MX_DOTS_THREADS = 1024;  // k_mx_dots: one block
constexpr int MX_UPDATE_ROWS = 2;       // rows a thread of k_mx_update loads before the dot sums

// Counters of a fused group of machines (see GroupArgs) during one implicit solve.
struct GroupState {
    int outer_active;               // members whose refinement has not converged
    int inner_active;               // members whose inner FP32 CG of the current pass runs
    int passes;                     // refinement launches of the current solve
    int launches;                   // SpMV launches of the current pass
};

struct MixArgs;

// Block ranges of one fused launch: member m owns blocks [first[m], first[m + 1]).
struct GroupLaunch {
    const int* member;              // [blocks] member of each block
    const int* first;               // [members + 1]
};

// Fused FP32 CG of several machines of a batch (one launch per kernel over all members'
// blocks). Each member keeps its own MixArgs, block partition, partial sums and scalars,
// so that its arithmetic is that of its own launches; the loop conditions are shared and
// cleared when the last member stops.
struct GroupArgs {
    const MixArgs* args;            // [members] the members' arguments of this solve
    GroupLaunch spmv, update, refine;
    GroupState* gs;
    unsigned long long h_outer, h_inner;
    int tail_pairs;                 // (spmv, update) pairs after this one in the loop body
    int n_members;
    int launch_cap;                 // SpMV launches of a pass after which the inner loop stops
    int pass_cap;                   // refinement launches after which the outer loop stops
};

struct MixArgs {
    EllDev A;                       // val (FP64) for residuals, val32 for the inner solves
    const double* mass;
    const float* mass32;
    const double* diagK;
    double dtau;
    int64_t n;
    double *X, *R, *B;              // FP64 iterate, residual, right-hand side
    float *Dl, *Rl, *Ul, *Pl, *Wl, *Sl, *Dinv;   // FP32 correction, residual, u, direction, A u, A p, 1/diag
    float* Dsum;                    // FP32 sum of the corrections of all passes (x - x0)
    int* loop_kernels;              // StepState::loop_kernels
    CgState* cg;                    // inner scalars (bb holds the inner initial ||r||^2)
    MixState* ms;                   // outer scalars
    double* partials;
    double* gpartials;              // group totals of the two-level reduction
    unsigned int* counter;          // [0] groups done, [1 + g] blocks of group g done
    int* iters_out;                 // inner iterations of this solve (all passes)
    int* refine_out;                // refinement passes of this solve
    double* true_res;               // k_mx_true_residual: ||b - A x|| / ||b|| of this solve
    int* status;
    int defer;                      // 1: k_mx_spmv + k_mx_update (deferred dots), 0: k_mx_spmv +
                                    // k_mx_dots + k_mx_update_red4 (large grids)
    int pair_kernels;               // kernels of one CG iteration (2 or 3): launch counting
    int part_blocks;                // grid of k_mx_spmv: number of its block partials
    int max_iter;                   // per inner solve
    int tail_pairs;                 // (spmv, update) pairs after this one in the graph's loop body
    int max_refine;
    double rtol2;                   // outer: ||b - A x||^2 <= rtol2 ||b||^2
    double inner_rtol2;             // inner: ||r||^2 <= inner_rtol2 ||r_0||^2
    unsigned long long h_outer, h_inner;
    GroupState* grp;                // fused group the solve runs in, or NULL
};

// Right-hand side of the implicit stage.
struct RhsArgs {
    int mode;
    const double* b_in;             // RHS_GIVEN
    const double* Tprev;            // T_{m-1} of the current iterate
    const double* g;                // b_env
    const double* FIm;              // F^I(T^k_m) (sweep)
    const double* FI[MAX_M];        // F^I(T^k_j), j = 1..M (sweep)
    double Sdt[MAX_M];              // dt s_{m,j}
    int nFI;
    // contact-DOF term of the right-hand side, or NULL: sweep: sum_q dt shat_{m,q}
    // f^E(T^k_{m,q}); predictor: single-rate SDC's or implicit Euler's f^E part
    const double* ihat;
    const int32_t* pos;             // DOF -> contact index or -1
    const double* x0;               // initial guess
    // F^I(x0) + g if known (NULL: form m x0 + dtau K x0 with an SpMV). Then
    // m x0 + dtau K x0 = m x0 - dtau (F^I(x0) + g - g) needs no pass over K.
    const double* Fx0;
};

// Bulk endpoint update after the solve (see k_bulk_endpoint).
enum { BULK_ALL = 0, BULK_CONTACT = 1, BULK_OFF_CONTACT = 2 };

struct BulkArgs {
    EllDev A;
    const double* minv;
    const double* g;
    const double* X;                // T*
    const double* Tprev;
    double* Tout;
    const double* FIm;
    const double* FI[MAX_M];
    double Sdt[MAX_M];
    int nFI;
    double dtau;
    int mode;
    int64_t n;
    const int32_t* pos;             // DOF -> contact index or -1
    double* fstar_I;                // [NI] f*_m on the contact DOFs (output)
    // rows of this launch: BULK_ALL, BULK_CONTACT (one thread per contact DOF, through dof),
    // or BULK_OFF_CONTACT (every row not on the contact)
    int rows;
    const int32_t* dof;             // [NI] contact index -> DOF
    int n_iface;
    // mixed precision (k_bulk_endpoint_mx): T* = x0 + dX with dX the solve's accumulated FP32
    // correction, so K T* = K x0 + K dX with K x0 known through F^I(x0); the pass over K is
    // an FP32 SpMV of dX. The output increment T_m - T_{m-1} goes to dT (FP32).
    const float* dX;
    const double* Fx0;              // F^I(x0) + g (x0 = T_{m-1} in the predictor, T^k_m in a sweep)
    float* dT;
};

// F^I(T_m) + g = F^I(T_prev) + g - K (T_m - T_prev) with the increment dT in FP32 (mixed precision).
struct FiDevArgs {
    EllDev A;
    const double* Fprev;
    const float* dT;
    double* F;
    int64_t n;
};


struct GeomArgs {
    ContactDev C;
    CouplingOp E;
    const double* slot_pos;   // unit-step position of each slot (tau = t_n + dt pos)
    const StepState* st;      // t_n = st->t0 + st->n_done * dt
    double t_fixed;           // used instead of t_n + dt pos when use_fixed
    int use_fixed;
    int n_slots;
    int* status;
};

// T-independent part of every substep increment of one interval
// (Algorithm 1 / Algorithm 2 inner loops), on the contact DOFs:
//   predictor: c_p = dt_p f*_m
//   sweep:     c_p = dt_p (f*_m - f^E(T^k_{m,p-1})) + I_{m,p-1}^p,
//              I_{m,p-1}^p = sum_j dt stil_{m,p,j} F^I_j + sum_q dt s_{m,p,q} f^E(T^k_{m,q})
// so that m T_{m,p} = m T_{m,p-1} + c_p + dt_p f^E(T^{k+1}_{m,p-1}).
struct PrepArgs {
    ContactDev C;
    int mode;                       // RHS_PRED or RHS_SWEEP
    int P;
    double dt;
    const StepState* st;
    const double* emb;              // P+1 unit-step positions of this interval's embedded nodes
    const double* FI[MAX_M];
    int nFI;
    const double* Stil;             // [P][nFI] dt stil_{m,p,j}
    const double* Semb;             // [P][P]  dt s_{m,p,q}
    const double* fe_old;           // [(P+1)][NI] previous iterate (sweep)
    double* cpre;                   // [P][NI] output (Algorithm 2): c_p - dt_p f*_m
    // mixed precision: base_q = f^E(T_{m-1}, tau_{m,q}) for q = 0..P (output), from
    // the interval's slots of the coupling operator and T_{m-1} = Tprev
    double* base;                   // [(P+1)][NI] or NULL
    CouplingOp E;                   // indices are contact-DOF ids
    int slot0;
    const double* Tprev;
    const double* Tc;               // mixed: T_{m-1} on the contact DOFs, by contact index (k_iface_tc)
};

// Single-rate SDC on the contact DOFs: f^E at one slot, and the implicit stage's contact terms.
struct SisdcArgs {
    ContactDev C;
    CouplingOp E;                   // indices are contact-DOF ids
    // k_sisdc_fe
    const double* T;                // [n] temperature at the node
    int slot;
    double* fe_out;                 // [NI]
    // k_sisdc_rhs
    int mode;                       // RHS_PRED or RHS_SWEEP
    double dtau;
    const double* fe_left_new;      // [NI] f^E(T^{k+1}_{m-1}, tau_{m-1})
    const double* fe_left_old;      // [NI] f^E(T^k_{m-1}, tau_{m-1}) (sweep)
    const double* fe_old[MAX_M];    // [NI] f^E(T^k_j, tau_j), j = 1..M (sweep)
    double Sdt[MAX_M];              // dt s_{m,j}
    int nFE;
    double* ihat;                   // [NI] output
};

// Sequential substeps of one interval on the contact DOFs (one cluster).
struct IfaceArgs {
    ContactDev C;
    int mode;                       // RHS_PRED or RHS_SWEEP
    int first;                      // first non-degenerate interval of the step
    int P;
    double dt;
    const StepState* st;
    const double* emb;              // P+1 unit-step positions of this interval's embedded nodes
    const double* Tprev;            // T_{m-1} (N)
    double* Tout;                   // T_m (N), contact rows written here
    const double* cpre;             // [P][NI] c_p less dt_p f*_m (Algorithm 2; unread in Algorithm 1)
    const double* fstar;            // [NI] f*_m of the interval
    const double* Shat;             // [P]     dt shat_{m,q}
    CouplingOp E;                   // slots of this interval start at slot0
    int slot0;
    const double* fe_old;           // [(P+1)][NI] previous iterate (sweep)
    double* fe_new;                 // [(P+1)][NI]
    const double* fe_prev_end;      // [NI] this iterate's f^E at the end of the previous interval
    double* ihat_new;               // [NI]
    const double* base;             // mixed: [(P+1)][NI] f^E(T_{m-1}, tau_{m,q}) from k_iface_prep
    int chunk;                      // replica slots per CTA (the cluster size is the grid)
    float* dT;                      // mixed: T_m - T_{m-1} on the contact rows (output), or NULL
    void* rep_global;               // [2][cs * chunk] replica buffers of the global-replica loop
    int* status;                    // sticky status word (SDC_ERR_TIMEOUT if an exchange wait gives up)
    int* sent;                      // [IFACE_MAX_CLUSTER] chunks each CTA of the cluster sent (per launch)
    unsigned* gbar;                 // grid form: [count, generation] of its grid barrier (zeroed per launch)
    long long poll_limit;           // polls of an exchange wait before it gives up
};

// Polls of an exchange wait of the contact loop (sdc_set_wait_limit overrides it), and of
// the waits that drain the copies still addressed to a CTA after a wait gave up.
constexpr long long IFACE_POLLS = 1ll << 24;
constexpr long long IFACE_DRAIN_POLLS = 1ll << 24;

struct ResidualArgs {
    const double* mass;
    const double* Tn;
    const double* Tm[MAX_M];        // T^k_m, m = 1..M
    const double* FI[MAX_M];
    double Sdt[MAX_M][MAX_M];
    const double* ihat[MAX_M];      // per interval, NI values (NULL for a zero-length interval)
    const int32_t* pos;
    int M;
    int64_t n;
    double* partials;
    unsigned int* counter;
    double* out;
};

// kernels (defined in kernels.cu)
// Kernels that read the matrix come in both column forms of EllDev (32-bit columns, or 16-bit
// offsets from each slice's base); name##_form(c32) returns the one for a matrix.
using KEllOp = void (*)(EllDev, const double*, double, const double*, double*);
using KEllFi = void (*)(EllDev, const double*, const double*, double*, int*);
using KCgInit = void (*)(CgArgs, RhsArgs);
using KCg = void (*)(CgArgs);
using KMxInit = void (*)(MixArgs, RhsArgs);
using KMx = void (*)(MixArgs);
using KGroup = void (*)(GroupArgs);
using KBulk = void (*)(BulkArgs);
using KFi = void (*)(FiDevArgs);
KEllOp k_apply_operator_form(bool c32);
KEllFi k_fi_form(bool c32);
KCgInit k_cg_init_form(bool c32);
KCg k_cg_spmv_form(bool c32);
KCgInit k_ie_init_form(bool c32);
KCg k_ie_spmv_form(bool c32);
KMxInit k_mx_init_form(bool c32);
KMx k_mx_true_residual_form(bool c32);
KBulk k_bulk_endpoint_form(bool c32);
// The kernels that read only the FP32 copy of K: f = 0 (16-bit offsets), 1 (32-bit
// columns) or 2 (implied columns, EllDev::stab set).
KMx k_mx_spmv_form32(int f);
KMx k_mx_refine_form32(int f);
KGroup k_mx_spmv_g_form32(int f);
KGroup k_mx_refine_g_form32(int f);
KBulk k_bulk_endpoint_mx_form32(int f);
KFi k_fi_mx_form32(int f);
__global__ void k_sisdc_fe(SisdcArgs a);
__global__ void k_sisdc_rhs(SisdcArgs a);
__global__ void k_sisdc_endpoint(const double* X, const double* Tprev, double* Tout, float* dT, int64_t n);
__global__ void k_cg_update(CgArgs a);
__global__ void k_mx_update(MixArgs a);
__global__ void k_mx_update_red(MixArgs a);
__global__ void k_mx_dots(MixArgs a);
__global__ void k_mx_update_red4(MixArgs a);
__global__ void k_group_begin(GroupArgs g);
__global__ void k_group_end(GroupArgs g);
__global__ void k_mx_update_g(GroupArgs g);
__global__ void k_iface_geom(GeomArgs g);
__global__ void k_iface_geom_mx(GeomArgs g);
__global__ void k_contact_apply(ContactDev C, CouplingOp E, int slot, const double* T, double* Ti, double* out,
                                int phase);
__global__ void k_iface_prep(PrepArgs a);
__global__ void k_iface_tc(ContactDev C, const double* T, double* Tc);
__global__ void k_iface_loop(IfaceArgs a);
__global__ void k_iface_loop1(IfaceArgs a);
__global__ void k_iface_loop_gl(IfaceArgs a);
__global__ void k_iface_loop_mx(IfaceArgs a);
__global__ void k_iface_loop_mx1(IfaceArgs a);
__global__ void k_iface_loop_mx_gl(IfaceArgs a);
__global__ void k_iface_loop_gls(IfaceArgs a);
__global__ void k_iface_loop_grid(IfaceArgs a);
__global__ void k_iface_loop_mx_grid(IfaceArgs a);
constexpr int IFACE_GRID_THREADS = 256;  // threads per CTA of the grid-wide loop (one contact DOF each)
__global__ void k_iface_loop_mx_gls(IfaceArgs a);
__global__ void k_residual(ResidualArgs a);
__global__ void k_heat(const double* mass, const double* T, int64_t n, int64_t n_fix, double* partials,
                       unsigned int* counter, double* heat);
__global__ void k_step_end(StepState* st, const double* ihat, int n_int, int NI);

}  // namespace sdc
