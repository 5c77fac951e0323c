// C ABI of the GB300 IMEX multi-rate SDC heat solver: context, device
// memory, CUDA-graph construction of one macro step, and the entry points
// declared in sdcheat.h.
//
// One macro step (Algorithm 1 followed by K x Algorithm 2 of Sec. 3) is one
// CUDA graph. Each implicit solve is a conditional WHILE node whose body is
// one CG iteration; the last reduction of the iteration clears the
// condition once ||r|| <= rtol ||b|| or the iteration cap is hit, so a whole
// macro step runs without host round trips.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "kernels.cuh"

using namespace sdc;

namespace {
struct Chain;  // graph-node appender (below)
}

struct sdc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    sdc_alloc_fn alloc = nullptr;
    sdc_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::vector<void*> pool_asm, pool_scheme;
    std::vector<size_t> pool_asm_bytes, pool_scheme_bytes;

    // inputs
    BodyInput body[2];
    bool contact_set = false;
    std::vector<int64_t> cq_fix, cq_mov;
    double h_c = 0, q0 = 0;
    bool motion_set = false;
    double dir[3] = {0, 0, 1}, z0 = 0, amp = 0, period = 1;

    // assembled system
    bool assembled = false;
    int64_t n = 0, n_fix = 0, nnz = 0;
    HostCSR K;                      // concatenated, global column ids
    std::vector<double> mass_h, genv_h;
    EllDev A;
    double *d_mass = nullptr, *d_minv = nullptr, *d_diagK = nullptr, *d_genv = nullptr;
    ContactHost ch;
    ContactDev C;
    double* Tn = nullptr;
    StepState* st = nullptr;
    StepState* st_host = nullptr;   // pinned
    CgState* cgs = nullptr;
    double* partials = nullptr;
    double* gpartials = nullptr;    // group totals of the two-level reduction
    unsigned int* counter = nullptr;
    size_t n_counters = 0;
    unsigned update_grid = 1;       // grid of the deferred FP32 update (one wave)
    int update_bps = 0;             // sdc_set_update_blocks: its blocks per SM (0: as many as fit)
    double *X = nullptr, *R = nullptr, *U = nullptr, *P = nullptr, *Wv = nullptr, *S = nullptr, *D = nullptr;
    // mixed precision: FP64 right-hand side, FP32 inner vectors, FP32 mass, outer scalars
    double* Bv = nullptr;
    float *Dl = nullptr, *Rl = nullptr, *Ul = nullptr, *Pl = nullptr, *Wl = nullptr, *Sl = nullptr,
          *Dinv = nullptr;
    float* mass32 = nullptr;
    float* Dsum = nullptr;          // FP32 accumulated correction of the current solve (x - x0)
    float* dTv = nullptr;           // FP32 increment T_m - T_{m-1} of the current interval
    MixState* ms = nullptr;
    CouplingOp E1{};                // one slot, for sdc_contact_flux
    double* Ti1 = nullptr;
    int max_blocks = 0;
    int n_sms = 0;

    // scheme
    bool scheme_set = false;
    Weights W;
    int K_sweeps = 0;
    double dt = 1.0, rtol = 1e-12;
    int max_iter = 2000;
    int precision = SDC_FP64;
    int residuals = 0;
    int true_res = 0;               // sdc_set_diagnostics bit 1: FP64 true residual of mixed solves
    std::vector<int> nondeg;        // 1-based standard nodes m whose interval has positive length
    bool temp_set = false;

    // per-scheme device buffers
    std::vector<double*> Tstd;      // M+1, Tstd[0] = Tn
    double* FI[2][MAX_M] = {{nullptr}};
    double* Fn = nullptr;           // F^I(T_n) + g, formed once per macro step
    double* fe[2] = {nullptr, nullptr};
    double* ihat[2] = {nullptr, nullptr};
    double *cpre = nullptr, *fst = nullptr;
    double* fe_base = nullptr;      // mixed: f^E(T_{m-1}) at the interval's embedded nodes
    double* Tc = nullptr;           // mixed: T_{m-1} on the contact DOFs (k_iface_tc)
    int iface_cluster = 0;          // CTAs of the substep-loop cluster
    int iface_chunk = 0;            // replica slots per CTA of that cluster
    bool iface_global = false;      // replicas in global memory (large interfaces)
    bool iface_stage = false;       // global replicas staged in shared memory each substep
    bool iface_grid = false;        // grid-wide loop (sdc_set_contact_replicas 3): CTAs = iface_cluster
    unsigned* iface_gbar = nullptr; // its grid barrier's [count, generation]
    int force_global = 0;           // sdc_set_contact_replicas
    int max_cluster = 0;            // sdc_set_contact_cluster (0: automatic)
    int branches = 1;               // sdc_set_graph_branches
    int columns = 0;                // sdc_set_matrix_columns: 0 automatic, 16 = no implied, 32 = 32-bit
    bool c32 = false;               // the assembled matrix has 32-bit columns (else 16-bit offsets)
    bool implied = false;           // its FP32 copy has implied columns (ImpliedEll)
    int stepper = SDC_STEPPER_MRSDC;  // sdc_set_stepper
    int cg_unroll = 0;                // sdc_set_cg_unroll (0: by grid size)
    double* w_slot_ie = nullptr;      // implicit Euler: the unit position of t_{n+1} (one slot)
    double* ie_coef = nullptr;        // implicit Euler: FP64 coupling rows of that slot
    double* fe_std[2][MAX_M + 1] = {};  // single-rate SDC: f^E at the standard nodes, by iterate
    int in_batch = 0;               // batches holding this context (their members run without side branches)
    // set while a fused batch group emits this member's step: takes each mixed solve
    std::function<void(Chain&, MixArgs, const RhsArgs&)>* solve_hook = nullptr;
    void* iface_rep = nullptr;      // their buffers
    int* iface_sent = nullptr;      // chunks each CTA of the loop's cluster sent (per launch)
    long long poll_limit = IFACE_POLLS;  // sdc_set_wait_limit
    size_t iface_smem = 0;          // its dynamic shared memory per CTA
    CouplingOp E{};
    double *w_Stil = nullptr, *w_Semb = nullptr, *w_Shat = nullptr, *w_emb = nullptr, *w_slot = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_ready = false;
    bool buffers_ready = false;
    int fixed_kernels = 0;          // kernel nodes of the step graph outside the CG loops
    int eager = 0;                  // 1: plain launches, host-driven CG loop
    int eager_kernels = 0;          // kernels launched by the last eager step
    int* done_host = nullptr;       // pinned: CG iteration count, stop flag, SpMV runs
    bool own_stream = false;        // stream created by sdc_create_own_stream
    cudaEvent_t done_ev = nullptr;  // marks the copy of the CG stop flag (eager loop)

    // per-kernel device times of eager steps (CUDA events around each launch)
    int timing = 0;
    struct TimedLaunch {
        const void* f;
        int ev;                     // events ev (start) and ev + 1 (end) of ev_pool
        bool valid;
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<TimedLaunch> launches;
    std::vector<const void*> kind_f;            // accumulated per kernel
    std::vector<int> kind_n;
    std::vector<double> kind_ms;
};

namespace {

void* dalloc(sdc_ctx* c, std::vector<void*>& pool, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->user);
        if (!p) throw ApiError(SDC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw ApiError(SDC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
    }
    pool.push_back(p);
    (&pool == &c->pool_asm ? c->pool_asm_bytes : c->pool_scheme_bytes).push_back(bytes);
    return p;
}

// a kernel that reads the matrix, in the column form of the context's assembled matrix
#define MK(c, k) k##_form((c)->c32)
// the form of the FP32 copy: 2 = implied columns, else as the FP64 matrix
inline int form32(const sdc_ctx* c) { return c->implied ? 2 : c->c32 ? 1 : 0; }
#define MK32(c, k) k##_form32(form32(c))

template <class T>
T* dalloc_n(sdc_ctx* c, std::vector<void*>& pool, size_t count) {
    return static_cast<T*>(dalloc(c, pool, count * sizeof(T)));
}

template <class T>
T* upload(sdc_ctx* c, std::vector<void*>& pool, const std::vector<T>& v) {
    T* d = dalloc_n<T>(c, pool, v.size());
    if (!v.empty()) SDC_CUDA_TRY(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return d;
}

void free_pool(sdc_ctx* c, std::vector<void*>& pool) {
    if (pool.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (void* p : pool) {
        if (c->alloc) c->free_fn(p, c->user);
        else cudaFree(p);
    }
    pool.clear();
    (&pool == &c->pool_asm ? c->pool_asm_bytes : c->pool_scheme_bytes).clear();
}

void drop_graph(sdc_ctx* c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->graph_ready = false;
}

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Grid of a row kernel (blocks of RED_BLOCK threads): one row per thread.
// Measured on GB300 at 313k rows, grids of one wave with several rows per
// thread were no faster for the FP32 SpMV and slower for the FP64 one.
template <class F>
unsigned row_grid(sdc_ctx* c, F* kernel) {
    (void)kernel;
    return blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK);
}

// Appends nodes to a graph in a single dependency chain.
struct Chain {
    cudaGraph_t g;
    cudaGraphNode_t last = nullptr;
    int kernels = 0;
    cudaStream_t eager = nullptr;   // non-null: launch immediately instead of recording
    bool is_eager = false;
    sdc_ctx* timer = nullptr;       // eager only: record CUDA events around every launch
    std::vector<cudaGraphNode_t> joins;  // side branches the next node waits for as well
    bool allow_branches = true;          // false: side-branch kernels join the chain in place
    explicit Chain(cudaGraph_t gg) : g(gg) {}
    // dependencies of the next node on the chain: the last node and every pending join
    std::vector<cudaGraphNode_t> take_deps() {
        std::vector<cudaGraphNode_t> d;
        if (last) d.push_back(last);
        d.insert(d.end(), joins.begin(), joins.end());
        joins.clear();
        return d;
    }
    // The next node on the chain also waits for side-branch node n (graph mode; a
    // no-op in eager mode, where side-branch kernels were launched in stream order).
    void join(cudaGraphNode_t n) {
        if (n) joins.push_back(n);
    }
    // Side branch: a kernel node that waits only for `on` (null entries ignored), and
    // that the chain does not wait for until join(). Eager mode launches it at once.
    template <typename... KArgs>
    cudaGraphNode_t branch_kernel(std::initializer_list<cudaGraphNode_t> on, void (*f)(KArgs...), dim3 grid,
                                  dim3 block, KArgs... args) {
        if (is_eager || !allow_branches) {
            kernel_2d(f, grid, block, args...);
            return nullptr;
        }
        void* params[] = {(void*)&args...};
        ++kernels;
        std::vector<cudaGraphNode_t> d;
        for (cudaGraphNode_t n : on)
            if (n) d.push_back(n);
        cudaKernelNodeParams p{};
        p.func = (void*)f;
        p.gridDim = grid;
        p.blockDim = block;
        p.kernelParams = params;
        cudaGraphNode_t nd;
        SDC_CUDA_TRY(cudaGraphAddKernelNode(&nd, g, d.data(), d.size(), &p));
        return nd;
    }
    int begin_timed(const void* f) {
        if (!timer) return -1;
        const int ev = next_event();
        SDC_CUDA_TRY(cudaEventRecord(timer->ev_pool[ev], eager));
        timer->launches.push_back({f, ev, true});
        return ev;
    }
    void end_timed(int ev) {
        if (ev >= 0) SDC_CUDA_TRY(cudaEventRecord(timer->ev_pool[ev + 1], eager));
    }
    int next_event() {
        const int ev = 2 * (int)timer->launches.size();
        while ((int)timer->ev_pool.size() < ev + 2) {
            cudaEvent_t e;
            SDC_CUDA_TRY(cudaEventCreate(&e));
            timer->ev_pool.push_back(e);
        }
        return ev;
    }
    static Chain launcher(cudaStream_t s) {
        Chain c(nullptr);
        c.eager = s;
        c.is_eager = true;
        return c;
    }

    template <typename... KArgs>
    void kernel(void (*f)(KArgs...), unsigned grid, unsigned block, KArgs... args) {
        void* params[] = {(void*)&args...};
        ++kernels;
        if (is_eager) {
            const int ev = begin_timed((const void*)f);
            SDC_CUDA_TRY(cudaLaunchKernel((const void*)f, dim3(grid), dim3(block), params, 0, eager));
            end_timed(ev);
            return;
        }
        cudaKernelNodeParams p{};
        p.func = (void*)f;
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = 0;
        p.kernelParams = params;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddKernelNode(&nd, g, d.data(), d.size(), &p));
        last = nd;
    }
    template <typename... KArgs>
    void kernel_2d(void (*f)(KArgs...), dim3 grid, dim3 block, KArgs... args) {
        void* params[] = {(void*)&args...};
        ++kernels;
        if (is_eager) {
            const int ev = begin_timed((const void*)f);
            SDC_CUDA_TRY(cudaLaunchKernel((const void*)f, grid, block, params, 0, eager));
            end_timed(ev);
            return;
        }
        cudaKernelNodeParams p{};
        p.func = (void*)f;
        p.gridDim = grid;
        p.blockDim = block;
        p.kernelParams = params;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddKernelNode(&nd, g, d.data(), d.size(), &p));
        last = nd;
    }
    // Launch with dynamic shared memory and a thread-block cluster of `cluster` CTAs along x.
    template <typename... KArgs>
    void kernel_cluster(void (*f)(KArgs...), unsigned grid, unsigned block, size_t smem, unsigned cluster,
                        KArgs... args) {
        void* params[] = {(void*)&args...};
        ++kernels;
        if (is_eager) {
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(block);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = eager;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cluster;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            const int ev = begin_timed((const void*)f);
            SDC_CUDA_TRY(cudaLaunchKernelExC(&cfg, (const void*)f, params));
            end_timed(ev);
            return;
        }
        cudaKernelNodeParams p{};
        p.func = (void*)f;
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = (unsigned)smem;
        p.kernelParams = params;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddKernelNode(&nd, g, d.data(), d.size(), &p));
        cudaLaunchAttributeValue v{};
        v.clusterDim.x = cluster;
        v.clusterDim.y = 1;
        v.clusterDim.z = 1;
        SDC_CUDA_TRY(cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributeClusterDimension, &v));
        last = nd;
    }
    // cooperative launch (every block resident at once): kernels with a grid-wide barrier
    template <typename... KArgs>
    void kernel_coop(void (*f)(KArgs...), unsigned grid, unsigned block, KArgs... args) {
        void* params[] = {(void*)&args...};
        ++kernels;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        if (is_eager) {
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(block);
            cfg.stream = eager;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            const int ev = begin_timed((const void*)f);
            SDC_CUDA_TRY(cudaLaunchKernelExC(&cfg, (const void*)f, params));
            end_timed(ev);
            return;
        }
        cudaKernelNodeParams p{};
        p.func = (void*)f;
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.kernelParams = params;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddKernelNode(&nd, g, d.data(), d.size(), &p));
        SDC_CUDA_TRY(cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributeCooperative, &at[0].val));
        last = nd;
    }
    // zero `bytes` bytes of device memory (a memset node, or an async memset in eager mode)
    void zero(void* dst, size_t bytes) {
        if (is_eager) {
            SDC_CUDA_TRY(cudaMemsetAsync(dst, 0, bytes, eager));
            return;
        }
        cudaMemsetParams mp{};
        mp.dst = dst;
        mp.value = 0;
        mp.elementSize = 1;
        mp.width = bytes;
        mp.height = 1;
        mp.pitch = 0;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddMemsetNode(&nd, g, d.data(), d.size(), &mp));
        last = nd;
    }
    // event record node on the chain (graph mode only)
    void event(cudaEvent_t e) {
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddEventRecordNode(&nd, g, d.data(), d.size(), e));
        last = nd;
    }
    void copy(void* dst, const void* src, size_t bytes) {
        if (is_eager) {
            SDC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, eager));
            return;
        }
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddMemcpyNode1D(&nd, g, d.data(), d.size(), dst, src, bytes, cudaMemcpyDeviceToDevice));
        last = nd;
    }
    // WHILE node driven by handle h; returns the body graph.
    cudaGraph_t while_node(cudaGraphConditionalHandle h) {
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t nd;
        const std::vector<cudaGraphNode_t> d = take_deps();
        SDC_CUDA_TRY(cudaGraphAddNode(&nd, g, d.data(), nullptr, d.size(), &np));
        last = nd;
        return np.conditional.phGraph_out[0];
    }
};

CgArgs cg_args(sdc_ctx* c, double dtau, int solve_idx, double rtol, int max_iter) {
    CgArgs a{};
    a.A = c->A;
    a.mass = c->d_mass;
    a.diagK = c->d_diagK;
    a.dtau = dtau;
    a.n = c->n;
    a.X = c->X;
    a.R = c->R;
    a.U = c->U;
    a.P = c->P;
    a.W = c->Wv;
    a.S = c->S;
    a.D = c->D;
    a.cg = c->cgs;
    a.loop_kernels = &c->st->loop_kernels;
    a.partials = c->partials;
    a.gpartials = c->gpartials;
    a.counter = c->counter;
    a.iters_out = &c->st->cg_iters[solve_idx];
    a.status = &c->st->status;
    a.max_iter = max_iter;
    a.rtol2 = rtol * rtol;
    a.handle = 0;
    return a;
}

// Host-driven CG iterations (eager execution) with one iteration of lookahead:
// iteration j+1 is queued before the stop flag after iteration j is examined,
// so the GPU never waits for the host; an iteration queued after convergence
// finds the flag set and returns at once. An `iteration` here is one body of
// the graph's loop: `pairs` (SpMV, update) pairs of `pair_kernels` launches, each counting a
// run in CgState::runs when it works. Bodies that did no work are neither counted
// nor timed; the pairs after the stop within the last body are, as in the graph.
template <class Iter>
void eager_cg_loop(sdc_ctx* c, Chain& ch, Iter iteration, int pairs, int pair_kernels = 2) {
    const int KPI = pair_kernels * pairs;  // kernels per iteration
    iteration();
    int queued = 1;
    for (;;) {
        // iter, done and runs are adjacent in CgState: one copy of all three
        SDC_CUDA_TRY(cudaMemcpyAsync(c->done_host, &c->cgs->iter, 3 * sizeof(int), cudaMemcpyDeviceToHost, ch.eager));
        SDC_CUDA_TRY(cudaEventRecord(c->done_ev, ch.eager));
        iteration();
        ++queued;
        SDC_CUDA_TRY(cudaEventSynchronize(c->done_ev));
        if (c->done_host[1]) break;
    }
    // the first body always counts: in a pass with nothing to solve it only stops the loop
    const int idle = queued - std::max(1, (c->done_host[2] + pairs - 1) / pairs);
    ch.kernels -= KPI * idle;
    if (ch.timer)
        for (size_t k = ch.timer->launches.size() - (size_t)KPI * idle; k < ch.timer->launches.size(); ++k)
            ch.timer->launches[k].valid = false;
}

// Mixed precision: init, then WHILE_outer { inner init, WHILE_inner { spmv, update, p-update }, refine }
// (SpMV, update) pairs in one body of a CG loop. The WHILE node checks its
// condition and relaunches the body once per body; measured at 313k DOF, a
// body of three iterations makes the mixed macro step 2.5 % shorter than a
// body of one. A solve that stops early in a body leaves the body's later
// pairs to return at once, which costs more than it saves on grids of many
// blocks (5.75M DOF: 22k blocks a launch), so large grids keep one pair.
// (SpMV, update) pairs per body of a CG WHILE loop: more pairs cost fewer loop
// iterations (conditional-node evaluations) and more launches that find the solve
// stopped; sdc_set_cg_unroll overrides the default
int cg_unroll(sdc_ctx* c) {
    if (c->cg_unroll > 0) return c->cg_unroll;
    return blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK) <= (unsigned)MIX_DEFER_MAX_BLOCKS ? 3 : 1;
}

// The FP32 CG pair of a mixed solve: the deferred-dot SpMV and update on small grids, else
// the SpMV, one block that reduces its partials (k_mx_dots), and the update of four rows a thread (one a thread if a vector is not
// 16-byte aligned, as a user allocator's blocks may be).
void mx_spmv_launch(sdc_ctx* c, Chain& ch, const MixArgs& a) {
    ch.kernel(MK32(c, k_mx_spmv), row_grid(c, MK32(c, k_mx_spmv)), RED_BLOCK, a);
    if (!a.defer) ch.kernel(k_mx_dots, 1u, (unsigned)MX_DOTS_THREADS, a);
}

void mx_update_launch(sdc_ctx* c, Chain& ch, const MixArgs& a) {
    if (a.defer) {
        ch.kernel(k_mx_update, c->update_grid, RED_BLOCK, a);
        return;
    }
    bool aligned = true;
    for (const float* p : {a.Ul, a.Wl, a.Rl, a.Dinv, a.Pl, a.Sl, a.Dl}) aligned = aligned && (uintptr_t)p % 16 == 0;
    if (aligned) ch.kernel(k_mx_update_red4, (unsigned)blocks_for((c->n + 3) / 4, RED_BLOCK), RED_BLOCK, a);
    else ch.kernel(k_mx_update_red, row_grid(c, k_mx_update), RED_BLOCK, a);
}

void add_solve_mixed(sdc_ctx* c, Chain& ch, MixArgs a, const RhsArgs& r) {
    const int unroll = cg_unroll(c);
    if (ch.is_eager) {
        a.h_outer = a.h_inner = 0;
        ch.kernel(MK(c, k_mx_init), row_grid(c, MK(c, k_mx_init)), RED_BLOCK, a, r);
        for (;;) {
            SDC_CUDA_TRY(cudaMemcpyAsync(c->done_host, &c->ms->passes, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                         ch.eager));
            SDC_CUDA_TRY(cudaStreamSynchronize(ch.eager));
            if (c->done_host[1]) break;
            eager_cg_loop(
                c, ch,
                [&] {
                    for (int u = 0; u < unroll; ++u) {
                        mx_spmv_launch(c, ch, a);
                        mx_update_launch(c, ch, a);
                    }
                },
                unroll, a.pair_kernels);
            ch.kernel(MK32(c, k_mx_refine), row_grid(c, MK32(c, k_mx_refine)), RED_BLOCK, a);
        }
        return;
    }
    cudaGraphConditionalHandle ho;
    SDC_CUDA_TRY(cudaGraphConditionalHandleCreate(&ho, ch.g, 1u, cudaGraphCondAssignDefault));
    a.h_outer = (unsigned long long)ho;
    a.h_inner = 0;
    ch.kernel(MK(c, k_mx_init), row_grid(c, MK(c, k_mx_init)), RED_BLOCK, a, r);
    Chain outer(ch.while_node(ho));
    // the inner loop's condition: 1 at each graph launch (first pass), and set to 1 again by
    // k_mx_refine for every later pass
    cudaGraphConditionalHandle hi;
    SDC_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, outer.g, 1u, cudaGraphCondAssignDefault));
    a.h_inner = (unsigned long long)hi;
    Chain inner(outer.while_node(hi));
    for (int u = 0; u < unroll; ++u) {
        MixArgs au = a;
        au.tail_pairs = unroll - 1 - u;
        mx_spmv_launch(c, inner, au);
        mx_update_launch(c, inner, au);
    }
    outer.kernel(MK32(c, k_mx_refine), row_grid(c, MK32(c, k_mx_refine)), RED_BLOCK, a);
}

// init kernel, then WHILE { spmv, update, p-update }
void add_solve(sdc_ctx* c, Chain& ch, CgArgs a, const RhsArgs& r, void (*init)(CgArgs, RhsArgs) = nullptr,
               void (*spmv)(CgArgs) = nullptr) {
    if (!init) init = MK(c, k_cg_init);
    if (!spmv) spmv = MK(c, k_cg_spmv);
    const int unroll = cg_unroll(c);
    if (ch.is_eager) {
        a.handle = 0;
        ch.kernel(init, row_grid(c, MK(c, k_cg_init)), RED_BLOCK, a, r);
        eager_cg_loop(
            c, ch,
            [&] {
                for (int u = 0; u < unroll; ++u) {
                    ch.kernel(spmv, row_grid(c, MK(c, k_cg_spmv)), RED_BLOCK, a);
                    ch.kernel(k_cg_update, row_grid(c, k_cg_update), RED_BLOCK, a);
                }
            },
            unroll);
        return;
    }
    cudaGraphConditionalHandle h;
    SDC_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, ch.g, 1u, cudaGraphCondAssignDefault));
    a.handle = (unsigned long long)h;
    ch.kernel(init, row_grid(c, MK(c, k_cg_init)), RED_BLOCK, a, r);
    Chain body(ch.while_node(h));
    for (int u = 0; u < unroll; ++u) {
        CgArgs au = a;
        au.tail_pairs = unroll - 1 - u;
        body.kernel(spmv, row_grid(c, MK(c, k_cg_spmv)), RED_BLOCK, au);
        body.kernel(k_cg_update, row_grid(c, k_cg_update), RED_BLOCK, au);
    }
}

void require(bool ok, sdc_status code, const char* msg) {
    if (!ok) throw ApiError(code, msg);
}

constexpr double MIX_INNER_RTOL = 1e-6;   // FP32 inner solve: relative reduction per refinement pass
constexpr int MIX_INNER_MAX = 500;        // and its iteration cap per pass
constexpr int MIX_MAX_REFINE = 30;

MixArgs mix_args(sdc_ctx* c, double dtau, int solve_idx, double rtol, int max_iter) {
    MixArgs a{};
    a.A = c->A;
    a.mass = c->d_mass;
    a.mass32 = c->mass32;
    a.diagK = c->d_diagK;
    a.dtau = dtau;
    a.n = c->n;
    a.X = c->X;
    a.R = c->R;
    a.B = c->Bv;
    a.Dl = c->Dl;
    a.Rl = c->Rl;
    a.Ul = c->Ul;
    a.Pl = c->Pl;
    a.Wl = c->Wl;
    a.Sl = c->Sl;
    a.Dinv = c->Dinv;
    a.Dsum = c->Dsum;
    a.cg = c->cgs;
    a.ms = c->ms;
    a.loop_kernels = &c->st->loop_kernels;
    a.partials = c->partials;
    a.gpartials = c->gpartials;
    a.counter = c->counter;
    a.iters_out = &c->st->cg_iters[solve_idx];
    a.refine_out = &c->st->refinements[solve_idx];
    a.true_res = &c->st->true_res[solve_idx];
    a.status = &c->st->status;
    a.part_blocks = (int)row_grid(c, MK32(c, k_mx_spmv));
    a.defer = a.part_blocks <= MIX_DEFER_MAX_BLOCKS ? 1 : 0;
    a.pair_kernels = a.defer ? 2 : 3;
    a.max_iter = std::min(max_iter, MIX_INNER_MAX);
    a.max_refine = MIX_MAX_REFINE;
    a.rtol2 = rtol * rtol;
    a.inner_rtol2 = MIX_INNER_RTOL * MIX_INNER_RTOL;
    return a;
}

void add_implicit_solve(sdc_ctx* c, Chain& ch, double dtau, int solve_idx, double rtol, int max_iter,
                        const RhsArgs& r) {
    if (c->precision == SDC_MIXED_FP32) {
        const MixArgs a = mix_args(c, dtau, solve_idx, rtol, max_iter);
        if (c->solve_hook) {
            (*c->solve_hook)(ch, a, r);
            return;
        }
        add_solve_mixed(c, ch, a, r);
        if (c->true_res) ch.kernel(MK(c, k_mx_true_residual), row_grid(c, MK(c, k_mx_true_residual)), RED_BLOCK, a);
    } else {
        add_solve(c, ch, cg_args(c, dtau, solve_idx, rtol, max_iter), r);
    }
}


void build_ell(sdc_ctx* c) {
    const int64_t n = c->n;
    const int64_t ns = (n + SLICE - 1) / SLICE;
    std::vector<int64_t> sp(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t r = s * SLICE; r < std::min(n, (s + 1) * SLICE); ++r)
            w = std::max(w, c->K.row_ptr[r + 1] - c->K.row_ptr[r]);
        sp[s + 1] = sp[s] + w * SLICE;
    }
    std::vector<int32_t> col(sp[ns]);
    std::vector<double> val(sp[ns], 0.0);
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t w = (sp[s + 1] - sp[s]) / SLICE;
        for (int lane = 0; lane < SLICE; ++lane) {
            const int64_t r = s * SLICE + lane;
            const int64_t len = r < n ? c->K.row_ptr[r + 1] - c->K.row_ptr[r] : 0;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t o = sp[s] + k * SLICE + lane;
                if (k < len) {
                    col[o] = c->K.col[c->K.row_ptr[r] + k];
                    val[o] = c->K.val[c->K.row_ptr[r] + k];
                } else {
                    col[o] = (int32_t)std::min<int64_t>(r, n - 1);
                    val[o] = 0.0;
                }
            }
        }
    }
    c->A.n = n;
    c->A.n_slices = ns;
    c->A.slice_ptr = upload(c, c->pool_asm, sp);
    // 16-bit offsets from each slice's smallest column when every slice spans at most 65,535
    // columns (padding entries included: they hold a column of their slice), else 32-bit columns
    std::vector<int32_t> base(ns);
    bool narrow = c->columns != 32;
    for (int64_t s = 0; s < ns && narrow; ++s) {
        int32_t lo = INT32_MAX, hi = INT32_MIN;
        for (int64_t o = sp[s]; o < sp[s + 1]; ++o) {
            lo = std::min(lo, col[o]);
            hi = std::max(hi, col[o]);
        }
        base[s] = sp[s + 1] > sp[s] ? lo : 0;
        narrow = sp[s + 1] == sp[s] || (int64_t)hi - lo <= 65535;
    }
    c->c32 = !narrow;
    c->A.base = nullptr;
    c->A.off = nullptr;
    c->A.col = nullptr;
    if (narrow) {
        std::vector<uint16_t> off(sp[ns]);
        for (int64_t s = 0; s < ns; ++s)
            for (int64_t o = sp[s]; o < sp[s + 1]; ++o) off[o] = (uint16_t)(col[o] - base[s]);
        c->A.base = upload(c, c->pool_asm, base);
        c->A.off = upload(c, c->pool_asm, off);
    } else {
        c->A.col = upload(c, c->pool_asm, col);
    }
    c->A.val = upload(c, c->pool_asm, val);
    // the FP32 copy: implied columns when the matrix allows them (automatic form only), else
    // the layout of the FP64 values
    c->implied = false;
    c->A.slice_ptr32 = nullptr;
    c->A.stab = nullptr;
    c->A.stoff = nullptr;
    ImpliedEll ie;
    if (c->columns == 0 && build_implied_ell(c->K, ie)) {
        c->implied = true;
        c->A.slice_ptr32 = upload(c, c->pool_asm, ie.slice_ptr);
        c->A.stab = upload(c, c->pool_asm, ie.tab);
        c->A.stoff = upload(c, c->pool_asm, ie.off);
        c->A.val32 = upload(c, c->pool_asm, ie.val);
    } else {
        std::vector<float> v32(val.begin(), val.end());
        c->A.val32 = upload(c, c->pool_asm, v32);
    }
}

// One wave of the deferred FP32 update (rows strided): update_bps blocks a SM, or as many as
// fit, and no more blocks than 256-row groups. The update's sums do not depend on its grid.
void set_update_grid(sdc_ctx* c) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mx_update, RED_BLOCK, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    per_sm = std::max(per_sm, 1);
    if (c->update_bps > 0) per_sm = std::min(per_sm, c->update_bps);
    c->update_grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)per_sm * c->n_sms, blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK)));
}

void do_assemble(sdc_ctx* c) {
    require(c->body[0].set && c->body[1].set, SDC_ERR_STATE, "both bodies must be set before sdc_assemble");
    require(c->contact_set, SDC_ERR_STATE, "sdc_set_contact must precede sdc_assemble");
    require(c->motion_set, SDC_ERR_STATE, "sdc_set_motion must precede sdc_assemble");
    drop_graph(c);
    free_pool(c, c->pool_scheme);
    free_pool(c, c->pool_asm);
    c->assembled = false;
    c->temp_set = false;
    c->buffers_ready = false;

    HostCSR K0, K1;
    std::vector<double> m0, m1, g0, g1;
    assemble_body(c->body[0], K0, m0, g0);
    assemble_body(c->body[1], K1, m1, g1);
    const int64_t nf = K0.n, nm = K1.n;
    c->n_fix = nf;
    c->n = nf + nm;
    require(c->n < (int64_t)INT32_MAX, SDC_ERR_ARG, "too many DOFs");
    c->K.n = c->n;
    c->K.row_ptr.assign(c->n + 1, 0);
    c->K.col.resize(K0.col.size() + K1.col.size());
    c->K.val.resize(K0.val.size() + K1.val.size());
    std::copy(K0.row_ptr.begin(), K0.row_ptr.end(), c->K.row_ptr.begin());
    for (int64_t i = 1; i <= nm; ++i) c->K.row_ptr[nf + i] = K0.row_ptr[nf] + K1.row_ptr[i];
    std::copy(K0.col.begin(), K0.col.end(), c->K.col.begin());
    for (size_t k = 0; k < K1.col.size(); ++k) c->K.col[K0.col.size() + k] = K1.col[k] + (int32_t)nf;
    std::copy(K0.val.begin(), K0.val.end(), c->K.val.begin());
    std::copy(K1.val.begin(), K1.val.end(), c->K.val.begin() + K0.val.size());
    c->nnz = (int64_t)c->K.col.size();
    c->mass_h = m0;
    c->mass_h.insert(c->mass_h.end(), m1.begin(), m1.end());
    c->genv_h = g0;
    c->genv_h.insert(c->genv_h.end(), g1.begin(), g1.end());
    std::vector<double> diag(c->n, 0.0), minv(c->n);
    for (int64_t i = 0; i < c->n; ++i) {
        for (int64_t k = c->K.row_ptr[i]; k < c->K.row_ptr[i + 1]; ++k)
            if (c->K.col[k] == i) diag[i] = c->K.val[k];
        require(c->mass_h[i] > 0.0, SDC_ERR_ARG, "node with zero lumped mass (unused node?)");
        minv[i] = 1.0 / c->mass_h[i];
    }

    c->ch = build_contact(c->body[0], c->body[1], c->cq_fix, c->cq_mov, c->dir);

    SDC_CUDA_TRY(cudaSetDevice(c->device));
    build_ell(c);
    c->d_mass = upload(c, c->pool_asm, c->mass_h);
    c->d_minv = upload(c, c->pool_asm, minv);
    c->d_diagK = upload(c, c->pool_asm, diag);
    c->d_genv = upload(c, c->pool_asm, c->genv_h);

    // contact tables
    ContactHost& H = c->ch;
    ContactDev& C = c->C;
    C = ContactDev{};
    C.n_iface = (int)H.dof.size();
    require(C.n_iface <= IFACE_MAX_NI, SDC_ERR_ARG,
            "the contact interface has more than 32,768 DOFs (16 CTAs x 512 threads x 4 DOFs of the substep loop)");
    C.n_iface_fix = H.n_iface_fix;
    C.nq_fix = H.nq_fix;
    C.nq_mov = H.nq_mov;
    C.dof = upload(c, c->pool_asm, H.dof);
    std::vector<double> mI(H.dof.size());
    for (size_t a = 0; a < H.dof.size(); ++a) mI[a] = c->mass_h[H.dof[a]];
    C.mass = upload(c, c->pool_asm, mI);
    std::vector<double> mIinv(H.dof.size());
    for (size_t a = 0; a < H.dof.size(); ++a) mIinv[a] = minv[H.dof[a]];
    C.minv = upload(c, c->pool_asm, mIinv);
    std::vector<double> rinv(H.rect.size() / 2);
    for (size_t f = 0; f < H.rect.size() / 4; ++f) {
        rinv[2 * f + 0] = 1.0 / (H.rect[4 * f + 2] - H.rect[4 * f + 0]);
        rinv[2 * f + 1] = 1.0 / (H.rect[4 * f + 3] - H.rect[4 * f + 1]);
    }
    C.rinv = reinterpret_cast<const double2*>(upload(c, c->pool_asm, rinv));
    {
        // bounding boxes: per contact DOF (its faces) and per body (all its contact faces)
        std::vector<double> dbox((size_t)4 * C.n_iface);
        double bb[2][4] = {{1e300, 1e300, -1e300, -1e300}, {1e300, 1e300, -1e300, -1e300}};
        for (int a = 0; a < C.n_iface; ++a) {
            double b4[4] = {1e300, 1e300, -1e300, -1e300};
            for (int e = H.inc_ptr[a]; e < H.inc_ptr[a + 1]; ++e) {
                const double* r = &H.rect[4 * (size_t)H.inc_quad[e]];
                b4[0] = std::min(b4[0], r[0]);
                b4[1] = std::min(b4[1], r[1]);
                b4[2] = std::max(b4[2], r[2]);
                b4[3] = std::max(b4[3], r[3]);
            }
            double* bd = bb[a >= C.n_iface_fix ? 1 : 0];
            for (int k = 0; k < 4; ++k) dbox[4 * (size_t)a + k] = b4[k];
            bd[0] = std::min(bd[0], b4[0]);
            bd[1] = std::min(bd[1], b4[1]);
            bd[2] = std::max(bd[2], b4[2]);
            bd[3] = std::max(bd[3], b4[3]);
        }
        C.dof_box = reinterpret_cast<const Rect4*>(upload(c, c->pool_asm, dbox));
        C.box_fix = Rect4{bb[0][0], bb[0][1], bb[0][2], bb[0][3]};
        C.box_mov = Rect4{bb[1][0], bb[1][1], bb[1][2], bb[1][3]};
    }
    C.inc_ptr = upload(c, c->pool_asm, H.inc_ptr);
    C.inc_quad = upload(c, c->pool_asm, H.inc_quad);
    C.inc_code = upload(c, c->pool_asm, H.inc_code);
    C.rect = reinterpret_cast<const Rect4*>(upload(c, c->pool_asm, H.rect));
    C.qnode = reinterpret_cast<const int4*>(upload(c, c->pool_asm, H.qnode));
    auto bins = [&](const BinsHost& b) {
        BinsDev d;
        d.ou = b.ou;
        d.ov = b.ov;
        d.bu = b.bu;
        d.bv = b.bv;
        d.ibu = 1.0 / b.bu;
        d.ibv = 1.0 / b.bv;
        d.nu = b.nu;
        d.nv = b.nv;
        d.ptr = upload(c, c->pool_asm, b.ptr);
        d.item = upload(c, c->pool_asm, b.item);
        return d;
    };
    C.bins_fix = bins(H.bins_fix);
    C.bins_mov = bins(H.bins_mov);
    C.dir_u = H.dir_u;
    C.dir_v = H.dir_v;
    C.z0 = c->z0;
    C.amp = c->amp;
    C.period = c->period;
    C.q0 = c->q0;
    C.h_c = c->h_c;
    C.pos = upload(c, c->pool_asm, H.pos);

    // state and CG work vectors
    const size_t N = (size_t)c->n;
    c->Tn = dalloc_n<double>(c, c->pool_asm, N);
    c->X = dalloc_n<double>(c, c->pool_asm, N);
    c->R = dalloc_n<double>(c, c->pool_asm, N);
    c->U = dalloc_n<double>(c, c->pool_asm, N);
    c->P = dalloc_n<double>(c, c->pool_asm, N);
    c->Wv = dalloc_n<double>(c, c->pool_asm, N);
    c->S = dalloc_n<double>(c, c->pool_asm, N);
    c->D = dalloc_n<double>(c, c->pool_asm, N);
    c->Bv = dalloc_n<double>(c, c->pool_asm, N);
    c->Dl = dalloc_n<float>(c, c->pool_asm, N);
    c->Rl = dalloc_n<float>(c, c->pool_asm, N);
    c->Ul = dalloc_n<float>(c, c->pool_asm, N);
    c->Pl = dalloc_n<float>(c, c->pool_asm, N);
    c->Wl = dalloc_n<float>(c, c->pool_asm, N);
    c->Sl = dalloc_n<float>(c, c->pool_asm, N);
    c->Dsum = dalloc_n<float>(c, c->pool_asm, N);
    c->dTv = dalloc_n<float>(c, c->pool_asm, N);
    c->Dinv = dalloc_n<float>(c, c->pool_asm, N);
    {
        std::vector<float> m32(c->mass_h.begin(), c->mass_h.end());
        c->mass32 = upload(c, c->pool_asm, m32);
    }
    c->ms = dalloc_n<MixState>(c, c->pool_asm, 1);
    c->st = dalloc_n<StepState>(c, c->pool_asm, 1);
    c->cgs = dalloc_n<CgState>(c, c->pool_asm, 1);
    c->max_blocks = (int)blocks_for(c->n, RED_BLOCK) + 1;
    c->partials = dalloc_n<double>(c, c->pool_asm, (size_t)4 * c->max_blocks);
    const size_t n_groups = (size_t)c->max_blocks / 64 + 2;  // groups of the two-level reduction
    c->gpartials = dalloc_n<double>(c, c->pool_asm, 4 * n_groups);
    c->n_counters = 1 + n_groups;
    c->counter = dalloc_n<unsigned int>(c, c->pool_asm, c->n_counters);
    SDC_CUDA_TRY(cudaMemsetAsync(c->counter, 0, c->n_counters * sizeof(unsigned int), c->stream));
    set_update_grid(c);
    SDC_CUDA_TRY(cudaMemsetAsync(c->st, 0, sizeof(StepState), c->stream));
    const size_t NI = (size_t)C.n_iface;
    c->E1.cnt = dalloc_n<int32_t>(c, c->pool_asm, NI);
    c->E1.idx = dalloc_n<int32_t>(c, c->pool_asm, NI * MAXE);
    c->E1.coef = dalloc_n<double>(c, c->pool_asm, NI * MAXE);
    c->E1.cst = dalloc_n<double>(c, c->pool_asm, NI);
    c->Ti1 = dalloc_n<double>(c, c->pool_asm, NI);
    SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->assembled = true;
}

// The substep-loop kernel for a precision, a chunk size and the replica placement
// (one DOF per thread when the chunk fits the block; global replicas when two
// shared-memory replicas do not fit in a CTA).
using IfaceKernel = void (*)(IfaceArgs);
IfaceKernel iface_loop_kernel(bool mixed, int chunk, bool global, bool stage = false) {
    if (global && stage) return mixed ? k_iface_loop_mx_gls : k_iface_loop_gls;
    if (global) return mixed ? k_iface_loop_mx_gl : k_iface_loop_gl;
    const bool one = chunk <= IFACE_THREADS;
    if (mixed) return one ? k_iface_loop_mx1 : k_iface_loop_mx;
    return one ? k_iface_loop1 : k_iface_loop;
}

// Threads per CTA of that kernel: one warp-rounded thread per DOF of the chunk when
// it fits the block (no idle warps in the loop's barriers), else the full block.
int iface_loop_threads(int chunk, bool global) {
    if (global || chunk > IFACE_THREADS) return IFACE_THREADS;
    return std::max(32, (chunk + 31) & ~31);
}

// Cluster (16, 8, 4, 2 or 1 CTAs) of the substep loop: the preferred size below,
// else the first other size the device can co-schedule with room for every
// contact DOF. A CTA owns `chunk` replica slots: a multiple of 4 when the replicas
// live in shared memory (every chunk a whole number of 16-byte units for the bulk
// copies), of 32 in global memory (32-DOF tiles); shared memory when both buffers
// fit, else global memory. Without a cluster cap, an interface whose replicas fit no CTA
// takes the grid-wide loop instead when its CTAs fit the device.
void pick_iface_cluster(sdc_ctx* c) {
    const int NI = std::max(c->C.n_iface, 1);
    const bool mixed = c->precision == SDC_MIXED_FP32;
    const size_t esz = mixed ? sizeof(float) : sizeof(double);
    // dynamic shared memory a loop CTA may use: the device's opt-in limit per block less the
    // kernels' static shared memory (their mbarriers)
    int optin = 0;
    SDC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    size_t smem_cap = (size_t)optin;
    for (const void* k : {(const void*)k_iface_loop, (const void*)k_iface_loop1, (const void*)k_iface_loop_gl,
                          (const void*)k_iface_loop_mx, (const void*)k_iface_loop_mx1,
                          (const void*)k_iface_loop_mx_gl, (const void*)k_iface_loop_gls,
                          (const void*)k_iface_loop_mx_gls}) {
        cudaFuncAttributes fa{};
        SDC_CUDA_TRY(cudaFuncGetAttributes(&fa, k));
        smem_cap = std::min(smem_cap, (size_t)optin - fa.sharedSizeBytes);
    }
    for (const void* k : {(const void*)k_iface_loop, (const void*)k_iface_loop1, (const void*)k_iface_loop_gl,
                          (const void*)k_iface_loop_mx, (const void*)k_iface_loop_mx1,
                          (const void*)k_iface_loop_mx_gl, (const void*)k_iface_loop_gls,
                          (const void*)k_iface_loop_mx_gls}) {
        SDC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap));
        SDC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    c->iface_grid = false;
    // the grid-wide loop: one contact DOF a thread on as many co-resident CTAs as that takes
    auto use_grid = [&]() {
        const void* kern = mixed ? (const void*)k_iface_loop_mx_grid : (const void*)k_iface_loop_grid;
        const int blocks = (int)blocks_for(NI, IFACE_GRID_THREADS);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, IFACE_GRID_THREADS, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        if ((int64_t)per_sm * c->n_sms < blocks) return false;
        c->iface_grid = true;
        c->iface_global = true;
        c->iface_stage = false;
        c->iface_cluster = blocks;
        c->iface_chunk = NI;
        c->iface_smem = 0;
        c->iface_rep = dalloc(c, c->pool_scheme, 2 * (size_t)NI * esz);
        return true;
    };
    int cs_max = IFACE_MAX_CLUSTER;
    while (c->max_cluster > 0 && cs_max > c->max_cluster) cs_max /= 2;
    // Preferred size: about IFACE_TARGET_CHUNK contact DOFs per CTA. Measured on GB300
    // (intervals of 20 substeps): 440 DOFs ran fastest on 4 CTAs (36 us against 43 on 16),
    // 990 on 8 (56 against 64), 3,950 and 7,000 on 16. Then larger clusters (smaller chunks
    // fit more easily), then smaller ones.
    int pref = 1;
    while (pref < cs_max && (int64_t)pref * IFACE_TARGET_CHUNK < NI) pref *= 2;
    std::vector<int> order;
    for (int cs = pref; cs <= cs_max; cs *= 2) order.push_back(cs);
    for (int cs = pref / 2; cs >= 1; cs /= 2) order.push_back(cs);
    // Automatic placement (no cluster cap set): shared-memory replicas when both buffers fit a
    // CTA of some cluster, else the grid-wide loop. Measured on GB300 (5,751,586-DOF machine, 27,170 contact DOFs,
    // P = 40): 241 us an interval on 107 CTAs against 631 us for the 16-CTA cluster with
    // staged global replicas; with 3,950 contact DOFs the shared-memory cluster is faster
    // (69 us against 118).
    bool shared_fits = false;
    for (int cs : order) {
        const int chunk = ((NI + cs - 1) / cs + 3) & ~3;
        shared_fits = shared_fits || (chunk <= IFACE_THREADS * IFACE_PER_THREAD &&
                                      2 * (size_t)cs * chunk * esz <= smem_cap);
    }
    if ((c->force_global == 3 || (c->force_global == 0 && c->max_cluster == 0 && !shared_fits)) && use_grid())
        return;
    for (int cs : order) {
        int chunk = ((NI + cs - 1) / cs + 3) & ~3;
        size_t rep_bytes = 2 * (size_t)cs * chunk * esz;
        bool global;
        if (!c->force_global && chunk <= IFACE_THREADS * IFACE_PER_THREAD && rep_bytes <= smem_cap) {
            global = false;
        } else {
            chunk = (chunk + 31) & ~31;  // global replicas are owned in 32-DOF tiles
            rep_bytes = 2 * (size_t)cs * chunk * esz;
            if (chunk > IFACE_THREADS * IFACE_PER_THREAD_GL) continue;
            global = true;
        }
        // global replicas are staged in shared memory (one buffer) when it fits, unless
        // sdc_set_contact_replicas asked for the unstaged form
        const size_t stage_bytes = (size_t)cs * chunk * esz;
        const bool stage = global && c->force_global != 2 && stage_bytes <= smem_cap;
        const size_t smem = global ? (stage ? stage_bytes : 0) : rep_bytes;
        const void* kern = (const void*)iface_loop_kernel(mixed, chunk, global, stage);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(iface_loop_threads(chunk, global));
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) {
            c->iface_cluster = cs;
            c->iface_chunk = chunk;
            c->iface_smem = smem;
            c->iface_global = global;
            c->iface_stage = stage;
            c->iface_rep = global ? dalloc(c, c->pool_scheme, rep_bytes) : nullptr;
            return;
        }
        cudaGetLastError();
    }
    throw ApiError(SDC_ERR_CUDA, "no thread-block cluster for the contact substep loop fits on this device");
}

void alloc_scheme_buffers(sdc_ctx* c) {
    free_pool(c, c->pool_scheme);
    const Weights& W = c->W;
    const int M = W.M, P = W.P;
    const size_t N = (size_t)c->n, NI = (size_t)c->C.n_iface;
    const int n_int = (int)c->nondeg.size();
    c->Tstd.assign(M + 1, nullptr);
    c->Tstd[0] = c->Tn;
    for (int m = 1; m <= M; ++m) {
        const bool degenerate = std::find(c->nondeg.begin(), c->nondeg.end(), m) == c->nondeg.end();
        c->Tstd[m] = degenerate ? c->Tstd[m - 1] : dalloc_n<double>(c, c->pool_scheme, N);
    }
    c->Fn = dalloc_n<double>(c, c->pool_scheme, N);
    for (int s = 0; s < 2; ++s)
        for (int j = 0; j < M; ++j) {
            const bool degenerate = std::find(c->nondeg.begin(), c->nondeg.end(), j + 1) == c->nondeg.end();
            // a zero-length first interval: T_1 = T_n in every iterate
            c->FI[s][j] = degenerate ? c->Fn : dalloc_n<double>(c, c->pool_scheme, N);
        }
    for (int s = 0; s < 2; ++s) {
        c->fe[s] = dalloc_n<double>(c, c->pool_scheme, (size_t)n_int * (P + 1) * NI);
        c->ihat[s] = dalloc_n<double>(c, c->pool_scheme, (size_t)n_int * NI);
        SDC_CUDA_TRY(cudaMemsetAsync(c->ihat[s], 0, (size_t)n_int * NI * sizeof(double), c->stream));
    }
    // f^E at the standard nodes for single-rate SDC: the nodes up to the first interval's
    // left end hold f^E(T_n, t_n) in both iterates (one buffer); later nodes one per iterate
    {
        double* fe0 = dalloc_n<double>(c, c->pool_scheme, NI);
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j <= M; ++j)
                c->fe_std[s][j] = j < c->nondeg[0] ? fe0 : (s == 0 ? dalloc_n<double>(c, c->pool_scheme, NI) : nullptr);
        for (int j = c->nondeg[0]; j <= M; ++j) c->fe_std[1][j] = dalloc_n<double>(c, c->pool_scheme, NI);
    }
    c->iface_sent = dalloc_n<int>(c, c->pool_scheme, IFACE_MAX_CLUSTER);
    c->iface_gbar = dalloc_n<unsigned>(c, c->pool_scheme, 2);
    c->cpre = dalloc_n<double>(c, c->pool_scheme, (size_t)P * NI);
    c->fst = dalloc_n<double>(c, c->pool_scheme, NI);
    pick_iface_cluster(c);
    const size_t slots = (size_t)n_int * (P + 1);
    c->E.cnt = dalloc_n<int32_t>(c, c->pool_scheme, slots * NI);
    c->E.idx = dalloc_n<int32_t>(c, c->pool_scheme, slots * MAXE * NI);
    const bool mixed = c->precision == SDC_MIXED_FP32;
    c->E.coef = mixed ? nullptr : dalloc_n<double>(c, c->pool_scheme, slots * MAXE * NI);
    c->E.cst = dalloc_n<double>(c, c->pool_scheme, slots * NI);
    c->E.coef32 = mixed ? dalloc_n<float>(c, c->pool_scheme, slots * MAXE * NI) : nullptr;
    // implicit Euler forms one slot in FP64 in both precisions (its coupling is in the matrix)
    c->ie_coef = mixed ? dalloc_n<double>(c, c->pool_scheme, (size_t)MAXE * NI) : c->E.coef;
    c->fe_base = mixed ? dalloc_n<double>(c, c->pool_scheme, (size_t)(P + 1) * NI) : nullptr;
    c->Tc = mixed ? dalloc_n<double>(c, c->pool_scheme, std::max<size_t>(NI, 1)) : nullptr;
    // dt-scaled weights
    std::vector<double> Stil(W.Stil), Semb(W.Semb), Shat(W.Shat), slot_pos(slots);
    for (double& v : Stil) v *= c->dt;
    for (double& v : Semb) v *= c->dt;
    for (double& v : Shat) v *= c->dt;
    for (int ii = 0; ii < n_int; ++ii)
        for (int q = 0; q <= P; ++q) slot_pos[(size_t)ii * (P + 1) + q] = W.emb[(size_t)(c->nondeg[ii] - 1) * (P + 1) + q];
    c->w_Stil = upload(c, c->pool_scheme, Stil);
    c->w_Semb = upload(c, c->pool_scheme, Semb);
    c->w_Shat = upload(c, c->pool_scheme, Shat);
    c->w_emb = upload(c, c->pool_scheme, W.emb);
    c->w_slot = upload(c, c->pool_scheme, slot_pos);
    c->w_slot_ie = upload(c, c->pool_scheme, std::vector<double>{1.0});
    SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
}

void emit_step(sdc_ctx* c, Chain& ch) {
    const Weights& W = c->W;
    const int M = W.M, P = W.P, K = c->K_sweeps;
    const int NI = c->C.n_iface;
    const int n_int = (int)c->nondeg.size();
    const double dt = c->dt;

    // geometry of f^E at every embedded node of the step (independent of T)
    GeomArgs ga{};
    ga.C = c->C;
    ga.E = c->E;
    ga.slot_pos = c->w_slot;
    ga.st = c->st;
    ga.use_fixed = 0;
    ga.n_slots = n_int * (P + 1);
    const bool ie = c->stepper == SDC_STEPPER_IMPLICIT_EULER;
    if (ie) {  // implicit Euler: the coupling at t_{n+1} only, in FP64
        ga.slot_pos = c->w_slot_ie;
        ga.n_slots = 1;
        ga.E.coef = c->ie_coef;
        ga.E.coef32 = nullptr;
    }
    ga.status = &c->st->status;
    // side branch: nothing reads the coupling operator before the first interval's
    // k_iface_prep, so it forms while the first implicit solve runs
    const cudaGraphNode_t geom = ch.branch_kernel(
        {ch.last}, c->precision == SDC_MIXED_FP32 && !ie ? k_iface_geom_mx : k_iface_geom,
        dim3(blocks_for(NI, GEOM_THREADS), (unsigned)ga.n_slots), dim3(GEOM_THREADS), ga);

    // F^I(T_n) + g in FP64 (the only pass over K in FP64 of a mixed-precision step); a
    // standard node at t_n (Lobatto) shares it. It also zeroes the step's count of CG-loop
    // kernels (no kernel that counts runs before or beside it).
    ch.kernel(MK(c, k_fi), row_grid(c, MK(c, k_fi)), (unsigned)RED_BLOCK, c->A, (const double*)c->d_genv, (const double*)c->Tn, c->Fn,
              &c->st->loop_kernels);
    const bool mixed = c->precision == SDC_MIXED_FP32;
    // F^I + g at standard node j (0 = t_n) of iterate set s
    auto F_at = [&](int j, int set) -> const double* { return j == 0 ? c->Fn : c->FI[set][j - 1]; };
    // mixed precision forms F^I at the nodes from the previous node's value and an FP32 SpMV of
    // the increment; with the FP64 SDC residual enabled every F^I is a full FP64 pass instead
    const bool fi_increment = mixed && !c->residuals;
    auto fi = [&](int m, int set) {
        if (fi_increment) {
            FiDevArgs fa{};
            fa.A = c->A;
            fa.Fprev = F_at(m - 1, set);
            fa.dT = c->dTv;
            fa.F = c->FI[set][m - 1];
            fa.n = c->n;
            ch.kernel(MK32(c, k_fi_mx), row_grid(c, MK32(c, k_fi_mx)), (unsigned)RED_BLOCK, fa);
        } else {
            ch.kernel(MK(c, k_fi), row_grid(c, MK(c, k_fi)), (unsigned)RED_BLOCK, c->A, (const double*)c->d_genv,
                      (const double*)c->Tstd[m], c->FI[set][m - 1], (int*)nullptr);
        }
    };
    // The bulk endpoint in two launches: f*_m on the contact rows, which the substep loop
    // needs, then T_m (and its increment) off the contact as a side branch beside the loop,
    // which writes the contact rows. The returned branch node is joined after the loop.
    auto bulk = [&](BulkArgs& b, const double* Fx0) -> cudaGraphNode_t {
        b.dof = c->C.dof;
        b.n_iface = NI;
        if (mixed) {
            b.dX = c->Dsum;
            b.Fx0 = Fx0;
            b.dT = c->dTv;
        }
        auto kern = mixed ? MK32(c, k_bulk_endpoint_mx) : MK(c, k_bulk_endpoint);
        b.rows = BULK_CONTACT;
        ch.kernel(kern, blocks_for(std::max(NI, 1), 256), 256u, b);
        b.rows = BULK_OFF_CONTACT;
        return ch.branch_kernel({ch.last}, kern, dim3(row_grid(c, kern)), dim3(RED_BLOCK), b);
    };

    auto sdt_row = [&](int m, double* out) {
        for (int j = 0; j < MAX_M; ++j) out[j] = j < M ? dt * W.S[(size_t)(m - 1) * M + j] : 0.0;
    };
    int solve = 0;
    // k_iface_prep of interval ii (standard node m) as a side branch that waits for
    // `on` only: it reads T_{m-1}, the previous iterate and the coupling operator, not
    // the interval's implicit solve, and runs beside it; substeps() joins it
    auto prep = [&](int ii, int m, int mode, int set_old, std::initializer_list<cudaGraphNode_t> on) {
        PrepArgs pa{};
        pa.C = c->C;
        pa.mode = mode;
        pa.P = P;
        pa.dt = dt;
        pa.st = c->st;
        pa.emb = c->w_emb + (size_t)(m - 1) * (P + 1);
        for (int j = 0; j < M; ++j) pa.FI[j] = c->FI[set_old][j];
        pa.nFI = M;
        pa.Stil = c->w_Stil + (size_t)(m - 1) * P * M;
        pa.Semb = c->w_Semb + (size_t)(m - 1) * P * P;
        pa.fe_old = c->fe[set_old] + (size_t)ii * (P + 1) * NI;
        pa.cpre = c->cpre;
        pa.base = c->fe_base;
        pa.E = c->E;
        pa.slot0 = ii * (P + 1);
        pa.Tprev = c->Tstd[m - 1];
        pa.Tc = c->Tc;
        if (c->Tc) {  // mixed: the contact DOFs' T_{m-1} packed first, in the same branch
            const cudaGraphNode_t t = ch.branch_kernel(on, k_iface_tc, dim3(blocks_for(std::max<int64_t>(NI, 1), 256)),
                                                       dim3(256u), c->C, (const double*)c->Tstd[m - 1], c->Tc);
            return ch.branch_kernel({t}, k_iface_prep, dim3(blocks_for((int64_t)(P + 1) * NI, 256)), dim3(256u), pa);
        }
        return ch.branch_kernel(on, k_iface_prep, dim3(blocks_for((int64_t)(P + 1) * NI, 256)), dim3(256u), pa);
    };
    // the cluster loop of interval ii, after the bulk endpoint and the interval's prep
    auto substeps = [&](int ii, int m, int mode, int set_old, int set_new, cudaGraphNode_t prep_node) {
        ch.join(prep_node);
        IfaceArgs ia{};
        ia.C = c->C;
        ia.mode = mode;
        ia.first = ii == 0;
        ia.P = P;
        ia.dt = dt;
        ia.st = c->st;
        ia.emb = c->w_emb + (size_t)(m - 1) * (P + 1);
        ia.Tprev = c->Tstd[m - 1];
        ia.Tout = c->Tstd[m];
        ia.cpre = c->cpre;
        ia.fstar = c->fst;
        ia.Shat = c->w_Shat + (size_t)(m - 1) * P;
        ia.E = c->E;
        ia.slot0 = ii * (P + 1);
        ia.fe_old = c->fe[set_old] + (size_t)ii * (P + 1) * NI;
        ia.fe_new = c->fe[set_new] + (size_t)ii * (P + 1) * NI;
        ia.fe_prev_end = ii > 0 ? c->fe[set_new] + ((size_t)(ii - 1) * (P + 1) + P) * NI : nullptr;
        ia.ihat_new = c->ihat[set_new] + (size_t)ii * NI;
        ia.base = c->fe_base;
        ia.chunk = c->iface_chunk;
        ia.status = &c->st->status;
        ia.dT = c->precision == SDC_MIXED_FP32 ? c->dTv : nullptr;
        ia.rep_global = c->iface_rep;
        ia.sent = c->iface_sent;
        ia.gbar = c->iface_gbar;
        ia.poll_limit = c->poll_limit;
        if (c->iface_grid) {
            ch.zero(c->iface_gbar, 2 * sizeof(unsigned));
            ch.kernel_coop(c->precision == SDC_MIXED_FP32 ? k_iface_loop_mx_grid : k_iface_loop_grid,
                           (unsigned)c->iface_cluster, (unsigned)IFACE_GRID_THREADS, ia);
            return;
        }
        ch.kernel_cluster(iface_loop_kernel(c->precision == SDC_MIXED_FP32, c->iface_chunk, c->iface_global,
                                            c->iface_stage),
                          (unsigned)c->iface_cluster, (unsigned)iface_loop_threads(c->iface_chunk, c->iface_global),
                          c->iface_smem,
                          (unsigned)c->iface_cluster, ia);
    };
    auto residual = [&](int set, int k) {
        ResidualArgs ra{};
        ra.mass = c->d_mass;
        ra.Tn = c->Tn;
        for (int m = 1; m <= M; ++m) {
            ra.Tm[m - 1] = c->Tstd[m];
            ra.FI[m - 1] = c->FI[set][m - 1];
            for (int j = 0; j < M; ++j) ra.Sdt[m - 1][j] = dt * W.S[(size_t)(m - 1) * M + j];
            auto it = std::find(c->nondeg.begin(), c->nondeg.end(), m);
            ra.ihat[m - 1] = it == c->nondeg.end() ? nullptr
                                                   : c->ihat[set] + (size_t)(it - c->nondeg.begin()) * NI;
        }
        ra.pos = c->C.pos;
        ra.M = M;
        ra.n = c->n;
        ra.partials = c->partials;
        ra.counter = c->counter;
        ra.out = &c->st->residual[k];
        ch.kernel(k_residual, row_grid(c, k_residual), (unsigned)RED_BLOCK, ra);
    };

    int ledger_intervals = n_int;
    if (ie) {
        // ---- fully implicit Euler with the contact coupling in the matrix (Sec. 1, Sec. 5):
        // (m + dt (K - L_E(t_{n+1}))) T_{n+1} = m T_n + dt (g + cst(t_{n+1})), FP64 PCG
        ch.join(geom);
        const unsigned gi = blocks_for(std::max(NI, 1), 256);
        SisdcArgs a = {};
        a.C = c->C;
        a.E = ga.E;
        a.mode = RHS_PRED;
        a.dtau = dt;
        a.fe_left_new = c->E.cst;  // slot 0: dt cst(t_{n+1}) on the contact rows
        a.ihat = c->ihat[0];
        ch.kernel(k_sisdc_rhs, gi, 256u, a);
        RhsArgs r{};
        r.mode = RHS_PRED;
        r.Tprev = c->Tn;
        r.g = c->d_genv;
        r.x0 = c->Tn;
        r.pos = c->C.pos;
        r.ihat = c->ihat[0];
        CgArgs ca = cg_args(c, dt, 0, c->rtol, c->max_iter);
        ca.ie.pos = c->C.pos;
        ca.ie.dof = c->C.dof;
        ca.ie.E = ga.E;
        ca.ie.slot = 0;
        ca.ie.NI = NI;
        add_solve(c, ch, ca, r, MK(c, k_ie_init), MK(c, k_ie_spmv));
        ch.copy(c->Tstd[M], c->X, (size_t)c->n * sizeof(double));
        // the step's contact heat for the ledger: dt f^E(T_{n+1}, t_{n+1})
        SisdcArgs f = a;
        f.T = c->X;
        f.slot = 0;
        f.fe_out = c->fe_std[0][M];
        ch.kernel(k_sisdc_fe, gi, 256u, f);
        a.fe_left_new = c->fe_std[0][M];
        a.ihat = c->ihat[K & 1];
        ch.kernel(k_sisdc_rhs, gi, 256u, a);
        ledger_intervals = 1;
    } else if (c->stepper == SDC_STEPPER_SISDC) {
        // ---- single-rate semi-implicit SDC (Sec. 3): f^E only at the standard nodes, in the
        // right-hand side of each interval's implicit stage; no substeps
        auto sis = [&]() {
            SisdcArgs a{};
            a.C = c->C;
            a.E = c->E;
            return a;
        };
        const unsigned gi = blocks_for(std::max(NI, 1), 256);
        // f^E(T, tau) at the slot of a standard node (an end slot of an interval)
        auto fe_at = [&](const double* T, int slot, double* out) {
            SisdcArgs a = sis();
            a.T = T;
            a.slot = slot;
            a.fe_out = out;
            ch.kernel(k_sisdc_fe, gi, 256u, a);
        };
        auto endpoint = [&](int m) {
            ch.kernel(k_sisdc_endpoint, row_grid(c, k_sisdc_endpoint), (unsigned)RED_BLOCK, (const double*)c->X,
                      (const double*)c->Tstd[m - 1], c->Tstd[m], mixed ? c->dTv : (float*)nullptr, (int64_t)c->n);
        };
        // f^E(T_n, t_n), the left node of the first interval in every iterate
        ch.join(geom);
        fe_at(c->Tn, 0, c->fe_std[0][c->nondeg[0] - 1]);
        for (int ii = 0; ii < n_int; ++ii) {
            const int m = c->nondeg[ii];
            const double dtau = dt * (W.c[m] - W.c[m - 1]);
            SisdcArgs a = sis();
            a.mode = RHS_PRED;
            a.dtau = dtau;
            a.fe_left_new = c->fe_std[0][m - 1];
            a.ihat = c->ihat[0] + (size_t)ii * NI;
            ch.kernel(k_sisdc_rhs, gi, 256u, a);
            RhsArgs r{};
            r.mode = RHS_PRED;
            r.Tprev = c->Tstd[m - 1];
            r.g = c->d_genv;
            r.x0 = c->Tstd[m - 1];
            r.Fx0 = F_at(m - 1, 0);
            r.pos = c->C.pos;
            r.ihat = a.ihat;
            add_implicit_solve(c, ch, dtau, solve++, c->rtol, c->max_iter, r);
            endpoint(m);
            fe_at(c->Tstd[m], ii * (P + 1) + P, c->fe_std[0][m]);
            fi(m, 0);
        }
        for (int k = 1; k <= K; ++k) {
            const int so = (k - 1) & 1, sn = k & 1;
            for (int ii = 0; ii < n_int; ++ii) {
                const int m = c->nondeg[ii];
                const double dtau = dt * (W.c[m] - W.c[m - 1]);
                SisdcArgs a = sis();
                a.mode = RHS_SWEEP;
                a.dtau = dtau;
                a.fe_left_new = c->fe_std[sn][m - 1];
                a.fe_left_old = c->fe_std[so][m - 1];
                for (int j = 0; j < M; ++j) a.fe_old[j] = c->fe_std[so][j + 1];
                sdt_row(m, a.Sdt);
                a.nFE = M;
                a.ihat = c->ihat[0] + (size_t)ii * NI;
                ch.kernel(k_sisdc_rhs, gi, 256u, a);
                RhsArgs r{};
                r.mode = RHS_SWEEP;
                r.Tprev = c->Tstd[m - 1];
                r.g = c->d_genv;
                r.FIm = c->FI[so][m - 1];
                for (int j = 0; j < M; ++j) r.FI[j] = c->FI[so][j];
                sdt_row(m, r.Sdt);
                r.nFI = M;
                r.ihat = a.ihat;
                r.pos = c->C.pos;
                r.x0 = c->Tstd[m];
                r.Fx0 = c->FI[so][m - 1];
                add_implicit_solve(c, ch, dtau, solve++, c->rtol, c->max_iter, r);
                endpoint(m);
                fe_at(c->Tstd[m], ii * (P + 1) + P, c->fe_std[sn][m]);
                if (k < K) fi(m, sn);
            }
        }
        // the contact heat of the step for the ledger (k_step_end): the quadrature
        // sum_j dt s_{m,j} f^E(T_j, tau_j) of the final iterate, per interval
        const int fin = K & 1;
        for (int ii = 0; ii < n_int; ++ii) {
            const int m = c->nondeg[ii];
            SisdcArgs a = sis();
            a.mode = RHS_SWEEP;
            a.dtau = 0.0;
            a.fe_left_new = a.fe_left_old = c->fe_std[fin][m - 1];
            for (int j = 0; j < M; ++j) a.fe_old[j] = c->fe_std[fin][j + 1];
            sdt_row(m, a.Sdt);
            a.nFE = M;
            a.ihat = c->ihat[K & 1] + (size_t)ii * NI;
            ch.kernel(k_sisdc_rhs, gi, 256u, a);
        }
    } else {
        // ---- Algorithm 1 (predictor)
        for (int ii = 0; ii < n_int; ++ii) {
            const int m = c->nondeg[ii];
            const double dtau = dt * (W.c[m] - W.c[m - 1]);
            const cudaGraphNode_t pn = prep(ii, m, RHS_PRED, 0, {ch.last, ii == 0 ? geom : nullptr});
            RhsArgs r{};
            r.mode = RHS_PRED;
            r.Tprev = c->Tstd[m - 1];
            r.g = c->d_genv;
            r.x0 = c->Tstd[m - 1];
            r.Fx0 = F_at(m - 1, 0);
            r.pos = c->C.pos;
            add_implicit_solve(c, ch, dtau, solve++, c->rtol, c->max_iter, r);
            BulkArgs b{};
            b.A = c->A;
            b.minv = c->d_minv;
            b.g = c->d_genv;
            b.X = c->X;
            b.Tprev = c->Tstd[m - 1];
            b.Tout = c->Tstd[m];
            b.dtau = dtau;
            b.mode = RHS_PRED;
            b.n = c->n;
            b.pos = c->C.pos;
            b.fstar_I = c->fst;
            const cudaGraphNode_t off = bulk(b, F_at(m - 1, 0));
            substeps(ii, m, RHS_PRED, 0, 0, pn);
            ch.join(off);
            fi(m, 0);
        }
        // ---- Algorithm 2 (sweeps)
        for (int k = 1; k <= K; ++k) {
            const int so = (k - 1) & 1, sn = k & 1;
            if (c->residuals) residual(so, k - 1);
            for (int ii = 0; ii < n_int; ++ii) {
                const int m = c->nondeg[ii];
                const double dtau = dt * (W.c[m] - W.c[m - 1]);
                const cudaGraphNode_t pn = prep(ii, m, RHS_SWEEP, so, {ch.last});
                RhsArgs r{};
                r.mode = RHS_SWEEP;
                r.Tprev = c->Tstd[m - 1];
                r.g = c->d_genv;
                r.FIm = c->FI[so][m - 1];
                for (int j = 0; j < M; ++j) r.FI[j] = c->FI[so][j];
                sdt_row(m, r.Sdt);
                r.nFI = M;
                r.ihat = c->ihat[so] + (size_t)ii * NI;
                r.pos = c->C.pos;
                r.x0 = c->Tstd[m];
                r.Fx0 = c->FI[so][m - 1];
                add_implicit_solve(c, ch, dtau, solve++, c->rtol, c->max_iter, r);
                BulkArgs b{};
                b.A = c->A;
                b.minv = c->d_minv;
                b.g = c->d_genv;
                b.X = c->X;
                b.Tprev = c->Tstd[m - 1];
                b.Tout = c->Tstd[m];
                b.FIm = c->FI[so][m - 1];
                for (int j = 0; j < M; ++j) b.FI[j] = c->FI[so][j];
                sdt_row(m, b.Sdt);
                b.nFI = M;
                b.dtau = dtau;
                b.mode = RHS_SWEEP;
                b.n = c->n;
                b.pos = c->C.pos;
                b.fstar_I = c->fst;
                const cudaGraphNode_t off = bulk(b, c->FI[so][m - 1]);
                substeps(ii, m, RHS_SWEEP, so, sn, pn);
                ch.join(off);
                if (k < K || c->residuals) fi(m, sn);
            }
        }
    }
    if (c->residuals) residual(K & 1, K);
    ch.copy(c->Tn, c->Tstd[M], (size_t)c->n * sizeof(double));
    ch.kernel(k_heat, row_grid(c, k_heat), (unsigned)RED_BLOCK, (const double*)c->d_mass, (const double*)c->Tn, (int64_t)c->n,
              (int64_t)c->n_fix, c->partials, c->counter, &c->st->heat[0]);
    ch.kernel(k_step_end, 1u, 256u, c->st, (const double*)c->ihat[K & 1], ledger_intervals, NI);
}

void build_step_graph(sdc_ctx* c) {
    drop_graph(c);
    SDC_CUDA_TRY(cudaGraphCreate(&c->graph, 0));
    Chain ch(c->graph);
    ch.allow_branches = c->branches && !c->in_batch;
    emit_step(c, ch);
    SDC_CUDA_TRY(cudaGraphInstantiate(&c->exec, c->graph, 0));
    c->fixed_kernels = ch.kernels;
    c->graph_ready = true;
}

sdc_status fail(sdc_ctx* c, sdc_status code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

template <class F>
sdc_status guarded(sdc_ctx* c, F&& f) {
    if (!c) return SDC_ERR_ARG;
    try {
        f();
        return SDC_OK;
    } catch (const ApiError& e) {
        return fail(c, e.code, e.what);
    } catch (const CudaError& e) {
        cudaGetLastError();
        return fail(c, e.code == cudaErrorMemoryAllocation ? SDC_ERR_OOM : SDC_ERR_CUDA, e.what);
    } catch (const std::bad_alloc&) {
        return fail(c, SDC_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(c, SDC_ERR_ARG, e.what());
    }
}

void fill_report(sdc_ctx* c, sdc_step_report* rep) {
    const StepState& s = *c->st_host;
    std::memset(rep, 0, sizeof(*rep));
    rep->t = s.t0 + (double)s.n_done * s.dt;
    const bool ie = c->stepper == SDC_STEPPER_IMPLICIT_EULER;
    rep->sweeps = ie ? 0 : c->K_sweeps;
    const int n_solves = ie ? 1 : (int)c->nondeg.size() * (c->K_sweeps + 1);
    rep->n_solves = n_solves;
    for (int i = 0; i < n_solves; ++i) {
        rep->cg_iters_total += s.cg_iters[i];
        rep->cg_iters_max = std::max(rep->cg_iters_max, s.cg_iters[i]);
        rep->refinements_total += s.refinements[i];
    }
    rep->status = s.status;
    // graph: kernels outside the loops + those the loop bodies ran (counted on the device)
    rep->kernel_launches = c->eager ? c->eager_kernels : c->fixed_kernels + s.loop_kernels;
    for (int k = 0; k <= SDC_MAX_SWEEPS; ++k) rep->residual[k] = (c->residuals && k <= c->K_sweeps) ? s.residual[k] : -1.0;
    rep->heat_stand = s.heat[0];
    rep->heat_stock = s.heat[1];
    rep->contact_cluster = c->iface_cluster;
    rep->true_residual_max = -1.0;
    if (c->true_res && c->precision == SDC_MIXED_FP32 && !ie)
        for (int i = 0; i < n_solves; ++i) rep->true_residual_max = std::max(rep->true_residual_max, s.true_res[i]);
}

sdc_status read_state(sdc_ctx* c, sdc_step_report* rep) {
    SDC_CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream));
    SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (rep) fill_report(c, rep);
    const int s = c->st_host->status;
    if (s != 0) {
        SDC_CUDA_TRY(cudaMemsetAsync(&c->st->status, 0, sizeof(int), c->stream));
        if (s == SDC_ERR_NOT_CONVERGED) throw ApiError(SDC_ERR_NOT_CONVERGED, "a CG solve reached cg_max_iter");
        if (s == SDC_ERR_ARG) throw ApiError(SDC_ERR_ARG, "contact operator has more than 32 entries per DOF");
        if (s == SDC_ERR_TIMEOUT)
            throw ApiError(SDC_ERR_TIMEOUT, "a bounded wait of the contact substep loop gave up");
        throw ApiError((sdc_status)s, "device reported an error");
    }
    return SDC_OK;
}

void ensure_ready(sdc_ctx* c) {
    require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
    require(c->scheme_set, SDC_ERR_STATE, "call sdc_set_scheme first");
    require(c->temp_set, SDC_ERR_STATE, "call sdc_set_temperature first");
    if (!c->buffers_ready) {
        drop_graph(c);
        alloc_scheme_buffers(c);
        c->buffers_ready = true;
    }
    if (!c->eager && !c->graph_ready) build_step_graph(c);
}

const char* kernel_name(const void* f) {
    static const std::pair<const void*, const char*> names[] = {
        {(const void*)k_cg_update, "k_cg_update"}, {(const void*)k_iface_geom, "k_iface_geom"},
        {(const void*)k_iface_geom_mx, "k_iface_geom_mx"}, {(const void*)k_iface_prep, "k_iface_prep"},
        {(const void*)k_iface_tc, "k_iface_tc"}, {(const void*)k_iface_loop, "k_iface_loop"},
        {(const void*)k_iface_loop_mx, "k_iface_loop_mx"}, {(const void*)k_iface_loop1, "k_iface_loop1"},
        {(const void*)k_iface_loop_mx1, "k_iface_loop_mx1"}, {(const void*)k_iface_loop_gl, "k_iface_loop_gl"},
        {(const void*)k_iface_loop_mx_gl, "k_iface_loop_mx_gl"}, {(const void*)k_iface_loop_gls, "k_iface_loop_gls"},
        {(const void*)k_iface_loop_mx_gls, "k_iface_loop_mx_gls"},
        {(const void*)k_iface_loop_grid, "k_iface_loop_grid"},
        {(const void*)k_iface_loop_mx_grid, "k_iface_loop_mx_grid"}, {(const void*)k_sisdc_fe, "k_sisdc_fe"},
        {(const void*)k_sisdc_rhs, "k_sisdc_rhs"}, {(const void*)k_sisdc_endpoint, "k_sisdc_endpoint"},
        {(const void*)k_residual, "k_residual"}, {(const void*)k_heat, "k_heat"},
        {(const void*)k_step_end, "k_step_end"}, {(const void*)k_mx_update, "k_mx_update"},
        {(const void*)k_mx_update_red, "k_mx_update_red"}, {(const void*)k_mx_update_red4, "k_mx_update_red"},
        {(const void*)k_mx_dots, "k_mx_dots"},
        {(const void*)k_cg_init_form(false), "k_cg_init"}, {(const void*)k_cg_init_form(true), "k_cg_init"},
        {(const void*)k_cg_spmv_form(false), "k_cg_spmv"}, {(const void*)k_cg_spmv_form(true), "k_cg_spmv"},
        {(const void*)k_bulk_endpoint_form(false), "k_bulk_endpoint"},
        {(const void*)k_bulk_endpoint_form(true), "k_bulk_endpoint"},
        {(const void*)k_ie_init_form(false), "k_ie_init"}, {(const void*)k_ie_init_form(true), "k_ie_init"},
        {(const void*)k_ie_spmv_form(false), "k_ie_spmv"}, {(const void*)k_ie_spmv_form(true), "k_ie_spmv"},
        {(const void*)k_fi_form(false), "k_fi"}, {(const void*)k_fi_form(true), "k_fi"},
        {(const void*)k_mx_init_form(false), "k_mx_init"}, {(const void*)k_mx_init_form(true), "k_mx_init"},
        {(const void*)k_mx_spmv_form32(0), "k_mx_spmv"}, {(const void*)k_mx_spmv_form32(1), "k_mx_spmv"},
        {(const void*)k_mx_spmv_form32(2), "k_mx_spmv"},
        {(const void*)k_mx_refine_form32(0), "k_mx_refine"}, {(const void*)k_mx_refine_form32(1), "k_mx_refine"},
        {(const void*)k_mx_refine_form32(2), "k_mx_refine"},
        {(const void*)k_mx_true_residual_form(false), "k_mx_true_residual"},
        {(const void*)k_mx_true_residual_form(true), "k_mx_true_residual"},
        {(const void*)k_bulk_endpoint_mx_form32(0), "k_bulk_endpoint_mx"},
        {(const void*)k_bulk_endpoint_mx_form32(1), "k_bulk_endpoint_mx"},
        {(const void*)k_bulk_endpoint_mx_form32(2), "k_bulk_endpoint_mx"},
        {(const void*)k_fi_mx_form32(0), "k_fi_mx"}, {(const void*)k_fi_mx_form32(1), "k_fi_mx"},
        {(const void*)k_fi_mx_form32(2), "k_fi_mx"},
    };
    for (const auto& n : names)
        if (n.first == f) return n.second;
    return "other";
}

// Wait for the timed launches of an eager step and add their durations to the per-kernel sums.
void collect_times(sdc_ctx* c) {
    SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (const auto& L : c->launches) {
        if (!L.valid) continue;
        float ms = 0.f;
        SDC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_pool[L.ev], c->ev_pool[L.ev + 1]));
        size_t k = 0;
        while (k < c->kind_f.size() && c->kind_f[k] != L.f) ++k;
        if (k == c->kind_f.size()) {
            c->kind_f.push_back(L.f);
            c->kind_n.push_back(0);
            c->kind_ms.push_back(0.0);
        }
        c->kind_n[k] += 1;
        c->kind_ms[k] += ms;
    }
    c->launches.clear();
}

// One macro step on the context's stream.
void launch_step(sdc_ctx* c) {
    if (c->eager) {
        Chain ch = Chain::launcher(c->stream);
        if (c->timing) ch.timer = c;
        emit_step(c, ch);
        c->eager_kernels = ch.kernels;
        if (c->timing) collect_times(c);
    } else {
        SDC_CUDA_TRY(cudaGraphLaunch(c->exec, c->stream));
    }
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

sdc_status sdc_create(sdc_ctx** out, int device, void* cuda_stream) {
    if (!out) return SDC_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SDC_ERR_CUDA;
    }
    sdc_ctx* c = new (std::nothrow) sdc_ctx();
    if (!c) return SDC_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaMallocHost((void**)&c->st_host, sizeof(StepState)) != cudaSuccess ||
        cudaMallocHost((void**)&c->done_host, 4 * sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SDC_ERR_CUDA;
    }
    std::memset(c->st_host, 0, sizeof(StepState));
    if (cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        c->n_sms = 1;
    }
    *out = c;
    return SDC_OK;
}

sdc_status sdc_create_own_stream(sdc_ctx** out, int device) {
    if (!out) return SDC_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SDC_ERR_CUDA;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return SDC_ERR_CUDA;
    }
    const sdc_status r = sdc_create(out, device, st);
    if (r != SDC_OK) {
        cudaStreamDestroy(st);
        return r;
    }
    (*out)->own_stream = true;
    return SDC_OK;
}

sdc_status sdc_get_stream(const sdc_ctx* cc, void** stream) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(stream != nullptr, SDC_ERR_ARG, "stream is NULL");
        *stream = (void*)c->stream;
    });
}

void sdc_destroy(sdc_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    drop_graph(c);
    free_pool(c, c->pool_scheme);
    free_pool(c, c->pool_asm);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->done_host) cudaFreeHost(c->done_host);
    if (c->done_ev) cudaEventDestroy(c->done_ev);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

const char* sdc_last_error(const sdc_ctx* c) { return c ? c->err.c_str() : "null context"; }

sdc_status sdc_scheme_weights(sdc_nodes nodes, int M, int P, int window, double* c, double* emb, double* S,
                              double* Shat, double* Stil, double* Semb) {
    try {
        if (!(nodes == SDC_NODES_EQUI_NOLEFT || nodes == SDC_NODES_RADAU_RIGHT || nodes == SDC_NODES_LOBATTO) ||
            M < 1 || M > MAX_M || P < 1 || P > MAX_P || window < 0 || window > P ||
            (nodes == SDC_NODES_LOBATTO && M < 2))
            return SDC_ERR_ARG;
        const Weights W = make_weights(nodes, M, P, window);
        auto out = [](const std::vector<double>& v, double* dst) {
            if (dst) std::copy(v.begin(), v.end(), dst);
        };
        out(W.c, c);
        out(W.emb, emb);
        out(W.S, S);
        out(W.Shat, Shat);
        out(W.Stil, Stil);
        out(W.Semb, Semb);
        return SDC_OK;
    } catch (...) {
        return SDC_ERR_ARG;
    }
}

sdc_status sdc_set_allocator(sdc_ctx* c, sdc_alloc_fn alloc, sdc_free_fn free_fn, void* user) {
    return guarded(c, [&] {
        require(!c->assembled, SDC_ERR_STATE, "allocator must be set before sdc_assemble");
        require((alloc == nullptr) == (free_fn == nullptr), SDC_ERR_ARG, "give both alloc and free, or neither");
        c->alloc = alloc;
        c->free_fn = free_fn;
        c->user = user;
    });
}

sdc_status sdc_set_body(sdc_ctx* c, int body, const double* xyz, int64_t n_nodes, const int64_t* hex8, int64_t n_hex,
                        const double* k_per_hex, double k, double rho, double cc) {
    return guarded(c, [&] {
        require(body == 0 || body == 1, SDC_ERR_ARG, "body must be 0 (stand) or 1 (stock)");
        require(xyz && hex8 && n_nodes > 0 && n_hex > 0, SDC_ERR_ARG, "empty mesh");
        require(rho > 0 && cc > 0, SDC_ERR_ARG, "rho and c must be positive");
        require(k_per_hex || k > 0, SDC_ERR_ARG, "conductivity must be positive");
        BodyInput& b = c->body[body];
        b.xyz.assign(xyz, xyz + 3 * n_nodes);
        b.hex8.assign(hex8, hex8 + 8 * n_hex);
        if (k_per_hex) {
            b.k_hex.assign(k_per_hex, k_per_hex + n_hex);
            for (double v : b.k_hex) require(v > 0, SDC_ERR_ARG, "conductivity must be positive");
        } else {
            b.k_hex.clear();
        }
        b.k = k;
        b.rho = rho;
        b.c = cc;
        b.set = true;
        c->assembled = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_robin(sdc_ctx* c, int body, const int64_t* quad4, int64_t n_faces, double h, double T_env) {
    return guarded(c, [&] {
        require(body == 0 || body == 1, SDC_ERR_ARG, "body must be 0 or 1");
        require(n_faces >= 0 && (n_faces == 0 || quad4), SDC_ERR_ARG, "bad face list");
        require(h >= 0, SDC_ERR_ARG, "h must be >= 0");
        BodyInput& b = c->body[body];
        b.robin.assign(1, BodyInput::RobinGroup{});
        b.robin[0].quads.assign(quad4, quad4 + 4 * n_faces);
        b.robin[0].h = h;
        b.robin[0].T_env = T_env;
        c->assembled = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_add_robin(sdc_ctx* c, int body, const int64_t* quad4, int64_t n_faces, double h, double T_env) {
    return guarded(c, [&] {
        require(body == 0 || body == 1, SDC_ERR_ARG, "body must be 0 or 1");
        require(n_faces >= 0 && (n_faces == 0 || quad4), SDC_ERR_ARG, "bad face list");
        require(h >= 0, SDC_ERR_ARG, "h must be >= 0");
        BodyInput::RobinGroup grp;
        grp.quads.assign(quad4, quad4 + 4 * n_faces);
        grp.h = h;
        grp.T_env = T_env;
        c->body[body].robin.push_back(std::move(grp));
        c->assembled = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_contact(sdc_ctx* c, const int64_t* sq, int64_t n_sq, const int64_t* kq, int64_t n_kq, double h_c,
                           double q0_peak) {
    return guarded(c, [&] {
        require(sq && kq && n_sq > 0 && n_kq > 0, SDC_ERR_ARG, "empty contact face list");
        require(h_c >= 0 && q0_peak >= 0, SDC_ERR_ARG, "h_c and q0 must be >= 0");
        c->cq_fix.assign(sq, sq + 4 * n_sq);
        c->cq_mov.assign(kq, kq + 4 * n_kq);
        c->h_c = h_c;
        c->q0 = q0_peak;
        c->contact_set = true;
        c->assembled = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_motion(sdc_ctx* c, const double dir[3], double z0, double amp, double period) {
    return guarded(c, [&] {
        require(dir != nullptr, SDC_ERR_ARG, "dir is NULL");
        require(period > 0, SDC_ERR_ARG, "period must be > 0 (inf for a resting stock)");
        const double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        require(nrm > 0 && std::isfinite(nrm), SDC_ERR_ARG, "bad motion direction");
        for (int i = 0; i < 3; ++i) c->dir[i] = dir[i];
        c->z0 = z0;
        c->amp = amp;
        c->period = period;
        c->motion_set = true;
        if (c->assembled) {
            c->C.z0 = z0;
            c->C.amp = amp;
            c->C.period = period;
            require(std::fabs(dir[c->ch.normal]) <= 1e-12, SDC_ERR_ARG, "motion direction leaves the contact plane");
            c->C.dir_u = dir[c->ch.u];
            c->C.dir_v = dir[c->ch.v];
            c->graph_ready = false;
        }
    });
}

sdc_status sdc_assemble(sdc_ctx* c) {
    return guarded(c, [&] { do_assemble(c); });
}

sdc_status sdc_set_scheme(sdc_ctx* c, sdc_nodes nodes, int M, int P, int sweeps, int window, double dt, double cg_rtol,
                          int cg_max_iter, sdc_precision precision) {
    return guarded(c, [&] {
        require(nodes == SDC_NODES_EQUI_NOLEFT || nodes == SDC_NODES_RADAU_RIGHT || nodes == SDC_NODES_LOBATTO,
                SDC_ERR_ARG, "unknown node family");
        require(M >= 1 && M <= MAX_M, SDC_ERR_ARG, "M out of range [1, 16]");
        require(P >= 1 && P <= MAX_P, SDC_ERR_ARG, "P out of range [1, 64]");
        require(sweeps >= 0 && sweeps <= SDC_MAX_SWEEPS, SDC_ERR_ARG, "sweeps out of range [0, 15]");
        require(window >= 0 && window <= P, SDC_ERR_ARG, "window out of range [0, P]");
        require(dt > 0 && std::isfinite(dt), SDC_ERR_ARG, "dt must be positive");
        require(cg_rtol > 0 && cg_rtol < 1, SDC_ERR_ARG, "cg_rtol must be in (0, 1)");
        require(cg_max_iter >= 1, SDC_ERR_ARG, "cg_max_iter must be >= 1");
        require(precision == SDC_FP64 || precision == SDC_MIXED_FP32, SDC_ERR_ARG, "unknown precision");
        require(!(nodes == SDC_NODES_LOBATTO && M < 2), SDC_ERR_ARG, "Lobatto needs M >= 2");
        c->W = make_weights(nodes, M, P, window);
        c->K_sweeps = sweeps;
        c->dt = dt;
        c->rtol = cg_rtol;
        c->max_iter = cg_max_iter;
        c->precision = precision;
        c->nondeg.clear();
        for (int m = 1; m <= M; ++m)
            if (c->W.c[m] > c->W.c[m - 1]) c->nondeg.push_back(m);
        c->scheme_set = true;
        c->graph_ready = false;
        c->buffers_ready = false;
        if (c->assembled) {
            c->st_host->dt = dt;
            SDC_CUDA_TRY(cudaMemcpyAsync(&c->st->dt, &c->st_host->dt, sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream));
            SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
        }
    });
}

sdc_status sdc_set_execution(sdc_ctx* c, int eager) {
    return guarded(c, [&] {
        c->eager = eager ? 1 : 0;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_contact_replicas(sdc_ctx* c, int global) {
    return guarded(c, [&] {
        require(global >= 0 && global <= 3, SDC_ERR_ARG, "replica placement is 0, 1, 2 or 3");
        c->force_global = global;
        c->buffers_ready = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_cg_unroll(sdc_ctx* c, int pairs) {
    return guarded(c, [&] {
        require(pairs >= 0 && pairs <= 8, SDC_ERR_ARG, "CG loop pairs out of range [0, 8]");
        c->cg_unroll = pairs;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_graph_branches(sdc_ctx* c, int on) {
    return guarded(c, [&] {
        c->branches = on ? 1 : 0;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_contact_cluster(sdc_ctx* c, int max_ctas) {
    return guarded(c, [&] {
        require(max_ctas >= 0 && max_ctas <= IFACE_MAX_CLUSTER, SDC_ERR_ARG, "max_ctas out of range");
        c->max_cluster = max_ctas;
        c->buffers_ready = false;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_update_blocks(sdc_ctx* c, int blocks_per_sm) {
    return guarded(c, [&] {
        require(blocks_per_sm >= 0 && blocks_per_sm <= 32, SDC_ERR_ARG, "blocks_per_sm out of range [0, 32]");
        c->update_bps = blocks_per_sm;
        if (c->assembled) set_update_grid(c);
        c->graph_ready = false;
    });
}

sdc_status sdc_set_wait_limit(sdc_ctx* c, int64_t polls) {
    return guarded(c, [&] {
        require(polls >= 0, SDC_ERR_ARG, "polls must be >= 0");
        c->poll_limit = polls == 0 ? IFACE_POLLS : (long long)polls;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_kernel_timing(sdc_ctx* c, int on) {
    return guarded(c, [&] {
        c->timing = on ? 1 : 0;
        c->launches.clear();
        c->kind_f.clear();
        c->kind_n.clear();
        c->kind_ms.clear();
    });
}

sdc_status sdc_get_kernel_times(sdc_ctx* c, int32_t capacity, const char** names, int32_t* launches,
                                double* ms_total, int32_t* n_kinds) {
    return guarded(c, [&] {
        require(n_kinds != nullptr, SDC_ERR_ARG, "n_kinds is NULL");
        const int n = (int)c->kind_f.size();
        *n_kinds = n;
        for (int k = 0; k < std::min(n, (int)capacity); ++k) {
            if (names) names[k] = kernel_name(c->kind_f[k]);
            if (launches) launches[k] = c->kind_n[k];
            if (ms_total) ms_total[k] = c->kind_ms[k];
        }
    });
}

sdc_status sdc_set_stepper(sdc_ctx* c, int stepper) {
    return guarded(c, [&] {
        require(stepper == SDC_STEPPER_MRSDC || stepper == SDC_STEPPER_SISDC ||
                    stepper == SDC_STEPPER_IMPLICIT_EULER,
                SDC_ERR_ARG, "unknown stepper");
        require(stepper == SDC_STEPPER_MRSDC || !c->residuals, SDC_ERR_ARG,
                "residual diagnostics are available with MRSDC only");
        c->stepper = stepper;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_diagnostics(sdc_ctx* c, int flags) {
    return guarded(c, [&] {
        require(flags >= 0 && flags <= 3, SDC_ERR_ARG, "diagnostics flags are 0..3");
        require(!(flags & 1) || c->stepper == SDC_STEPPER_MRSDC, SDC_ERR_ARG,
                "residual diagnostics are available with MRSDC only");
        c->residuals = flags & 1;
        c->true_res = (flags >> 1) & 1;
        c->graph_ready = false;
    });
}

sdc_status sdc_set_temperature(sdc_ctx* c, const double* T, double T_uniform, double t0) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        if (T) {
            SDC_CUDA_TRY(cudaMemcpyAsync(c->Tn, T, (size_t)c->n * sizeof(double), cudaMemcpyDefault, c->stream));
        } else {
            std::vector<double> v((size_t)c->n, T_uniform);
            SDC_CUDA_TRY(cudaMemcpyAsync(c->Tn, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
        }
        StepState* h = c->st_host;
        std::memset(h, 0, sizeof(StepState));
        h->t0 = t0;
        h->dt = c->scheme_set ? c->dt : 1.0;
        SDC_CUDA_TRY(cudaMemcpyAsync(c->st, h, sizeof(StepState), cudaMemcpyHostToDevice, c->stream));
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->temp_set = true;
    });
}

sdc_status sdc_step(sdc_ctx* c, sdc_step_report* rep) {
    return guarded(c, [&] {
        ensure_ready(c);
        launch_step(c);
        if (rep) read_state(c, rep);
    });
}

sdc_status sdc_run_horizon(sdc_ctx* c, int64_t n_steps, sdc_step_report* last) {
    return guarded(c, [&] {
        require(n_steps >= 0, SDC_ERR_ARG, "n_steps must be >= 0");
        ensure_ready(c);
        for (int64_t i = 0; i < n_steps; ++i) launch_step(c);
        read_state(c, last);
    });
}

sdc_status sdc_step_async(sdc_ctx* c, int64_t n_steps) {
    return guarded(c, [&] {
        require(n_steps >= 0, SDC_ERR_ARG, "n_steps must be >= 0");
        ensure_ready(c);
        for (int64_t i = 0; i < n_steps; ++i) launch_step(c);
    });
}

sdc_status sdc_get_footprint(const sdc_ctx* cc, int64_t* bytes) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(bytes != nullptr, SDC_ERR_ARG, "bytes is NULL");
        size_t t = 0;
        for (size_t b : c->pool_asm_bytes) t += b;
        for (size_t b : c->pool_scheme_bytes) t += b;
        *bytes = (int64_t)t;
    });
}

sdc_status sdc_synchronize(sdc_ctx* c) {
    return guarded(c, [&] {
        if (c->assembled) read_state(c, nullptr);
        else SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
}

sdc_status sdc_set_matrix_columns(sdc_ctx* c, int bits) {
    return guarded(c, [&] {
        require(bits == 0 || bits == 16 || bits == 32, SDC_ERR_ARG, "bits must be 0 (automatic), 16 or 32");
        c->columns = bits;
    });
}

sdc_status sdc_get_matrix_columns(const sdc_ctx* cc, int32_t* bits) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(bits != nullptr, SDC_ERR_ARG, "bits is null");
        *bits = c->c32 ? 32 : 16;
    });
}

sdc_status sdc_get_matrix_implied(const sdc_ctx* cc, int32_t* implied) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(implied != nullptr, SDC_ERR_ARG, "implied is null");
        *implied = c->implied ? 1 : 0;
    });
}

sdc_status sdc_get_sizes(const sdc_ctx* cc, int64_t* n_dof, int64_t* n_stand, int64_t* nnz, int64_t* n_contact) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        if (n_dof) *n_dof = c->n;
        if (n_stand) *n_stand = c->n_fix;
        if (nnz) *nnz = c->nnz;
        if (n_contact) *n_contact = c->C.n_iface;
    });
}

sdc_status sdc_get_temperature(sdc_ctx* c, double* out, int64_t n) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(out && n == c->n, SDC_ERR_ARG, "out must hold n_dof doubles");
        SDC_CUDA_TRY(cudaMemcpyAsync(out, c->Tn, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream));
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
}

sdc_status sdc_get_temperature_device(const sdc_ctx* cc, const double** dptr) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(dptr != nullptr, SDC_ERR_ARG, "dptr is NULL");
        *dptr = c->Tn;
    });
}

sdc_status sdc_get_heat_totals(sdc_ctx* c, sdc_heat* out) {
    return guarded(c, [&] {
        require(c->assembled && c->temp_set, SDC_ERR_STATE, "no state yet");
        require(out != nullptr, SDC_ERR_ARG, "out is NULL");
        read_state(c, nullptr);
        const StepState& s = *c->st_host;
        if (s.n_done == 0) {
            // no step taken yet: compute the stored heat on the host side of the copy
            std::vector<double> T((size_t)c->n);
            SDC_CUDA_TRY(cudaMemcpy(T.data(), c->Tn, T.size() * sizeof(double), cudaMemcpyDeviceToHost));
            double h0 = 0, h1 = 0;
            for (int64_t i = 0; i < c->n; ++i) (i < c->n_fix ? h0 : h1) += c->mass_h[i] * T[i];
            out->stored_stand = h0;
            out->stored_stock = h1;
        } else {
            out->stored_stand = s.heat[0];
            out->stored_stock = s.heat[1];
        }
        out->friction_in = s.friction_in;
        out->t = s.t0 + (double)s.n_done * s.dt;
    });
}

sdc_status sdc_get_system(const sdc_ctx* cc, int64_t* row_ptr, int64_t* col, double* val, double* mass, double* genv) {
    sdc_ctx* c = const_cast<sdc_ctx*>(cc);
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        if (row_ptr) std::copy(c->K.row_ptr.begin(), c->K.row_ptr.end(), row_ptr);
        if (col)
            for (size_t k = 0; k < c->K.col.size(); ++k) col[k] = c->K.col[k];
        if (val) std::copy(c->K.val.begin(), c->K.val.end(), val);
        if (mass) std::copy(c->mass_h.begin(), c->mass_h.end(), mass);
        if (genv) std::copy(c->genv_h.begin(), c->genv_h.end(), genv);
    });
}

sdc_status sdc_apply_operator(sdc_ctx* c, double dtau, const double* x, double* y) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(x && y, SDC_ERR_ARG, "null buffer");
        auto apply = MK(c, k_apply_operator);
        apply<<<row_grid(c, apply), RED_BLOCK, 0, c->stream>>>(c->A, c->d_mass, dtau, x, y);
        SDC_CUDA_TRY(cudaGetLastError());
    });
}

sdc_status sdc_solve(sdc_ctx* c, double dtau, const double* b, double* x, int32_t* iters) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(b && x, SDC_ERR_ARG, "null buffer");
        require(dtau >= 0, SDC_ERR_ARG, "dtau must be >= 0");
        const double rtol = c->scheme_set ? c->rtol : 1e-12;
        const int max_iter = c->scheme_set ? c->max_iter : 2000;
        cudaGraph_t g;
        SDC_CUDA_TRY(cudaGraphCreate(&g, 0));
        std::unique_ptr<CUgraph_st, decltype(&cudaGraphDestroy)> guard(g, &cudaGraphDestroy);
        Chain ch(g);
        RhsArgs r{};
        r.mode = RHS_GIVEN;
        r.b_in = b;
        r.x0 = x;
        r.pos = c->C.pos;
        add_implicit_solve(c, ch, dtau, 0, rtol, max_iter, r);
        ch.copy(x, c->X, (size_t)c->n * sizeof(double));
        cudaGraphExec_t ex;
        SDC_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
        cudaError_t e = cudaGraphLaunch(ex, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(ex);
        SDC_CUDA_TRY(e);
        int it = 0;
        SDC_CUDA_TRY(cudaMemcpy(&it, &c->st->cg_iters[0], sizeof(int), cudaMemcpyDeviceToHost));
        if (iters) *iters = it;
        read_state(c, nullptr);
    });
}

sdc_status sdc_time_cg_iterations(sdc_ctx* c, double dtau, int32_t n_iters, int32_t spmv_only, float* ms,
                                  float* ms_spmv) {
    return guarded(c, [&] {
        require(n_iters >= 1 && n_iters <= 4096, SDC_ERR_ARG, "n_iters must be in 1..4096");
        require(ms != nullptr, SDC_ERR_ARG, "ms is NULL");
        require(dtau > 0.0, SDC_ERR_ARG, "dtau must be positive");
        ensure_ready(c);
        // the implicit-stage system with b = g and x0 = T_n: a nonzero residual; negative
        // tolerances and no iteration cap keep every iteration working (no stop test passes)
        const bool mixed = c->precision == SDC_MIXED_FP32;
        MixArgs ma = mix_args(c, dtau, 0, 1.0, 1);
        ma.rtol2 = -1.0;
        ma.inner_rtol2 = -1.0;
        ma.max_iter = 1 << 30;
        ma.max_refine = 1 << 30;
        CgArgs ca = cg_args(c, dtau, 0, 1.0, 1 << 30);
        ca.rtol2 = -1.0;
        RhsArgs r{};
        r.mode = RHS_GIVEN;
        r.b_in = c->d_genv;
        r.x0 = c->Tn;
        r.pos = c->C.pos;
        // graph 0: the initial residual; graph 1: the iterations; graph 2 (ms_spmv): the same
        // iterations with event records around every SpMV
        const int n_graphs = ms_spmv ? 3 : 2;
        std::vector<cudaGraph_t> g(n_graphs, nullptr);
        std::vector<cudaGraphExec_t> ex(n_graphs, nullptr);
        std::vector<cudaEvent_t> ev;
        auto release = [&] {
            for (auto e : ex)
                if (e) cudaGraphExecDestroy(e);
            for (auto x : g)
                if (x) cudaGraphDestroy(x);
            for (auto e : ev) cudaEventDestroy(e);
        };
        try {
            for (int k = 0; k < n_graphs; ++k) SDC_CUDA_TRY(cudaGraphCreate(&g[k], 0));
            const int n_ev = 2 + (ms_spmv ? 2 * n_iters : 0);
            for (int k = 0; k < n_ev; ++k) {
                cudaEvent_t e;
                SDC_CUDA_TRY(cudaEventCreate(&e));
                ev.push_back(e);
            }
            Chain init(g[0]);
            if (mixed) init.kernel(MK(c, k_mx_init), row_grid(c, MK(c, k_mx_init)), RED_BLOCK, ma, r);
            else init.kernel(MK(c, k_cg_init), row_grid(c, MK(c, k_cg_init)), RED_BLOCK, ca, r);
            for (int gi = 1; gi < n_graphs; ++gi) {
                Chain body(g[gi]);
                for (int k = 0; k < n_iters; ++k) {
                    if (gi == 2) body.event(ev[2 + 2 * k]);
                    if (mixed) mx_spmv_launch(c, body, ma);
                    else body.kernel(MK(c, k_cg_spmv), row_grid(c, MK(c, k_cg_spmv)), RED_BLOCK, ca);
                    if (gi == 2) body.event(ev[3 + 2 * k]);
                    if (spmv_only) continue;
                    if (mixed)
                        mx_update_launch(c, body, ma);
                    else
                        body.kernel(k_cg_update, row_grid(c, k_cg_update), RED_BLOCK, ca);
                }
            }
            for (int k = 0; k < n_graphs; ++k) SDC_CUDA_TRY(cudaGraphInstantiate(&ex[k], g[k], 0));
            SDC_CUDA_TRY(cudaGraphLaunch(ex[0], c->stream));
            SDC_CUDA_TRY(cudaEventRecord(ev[0], c->stream));
            SDC_CUDA_TRY(cudaGraphLaunch(ex[1], c->stream));
            SDC_CUDA_TRY(cudaEventRecord(ev[1], c->stream));
            SDC_CUDA_TRY(cudaEventSynchronize(ev[1]));
            SDC_CUDA_TRY(cudaEventElapsedTime(ms, ev[0], ev[1]));
            if (ms_spmv) {  // the same iterations again from the same start, timed per SpMV
                SDC_CUDA_TRY(cudaGraphLaunch(ex[0], c->stream));
                SDC_CUDA_TRY(cudaGraphLaunch(ex[2], c->stream));
                SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
                double sum = 0.0;
                for (int k = 0; k < n_iters; ++k) {
                    float t = 0.f;
                    SDC_CUDA_TRY(cudaEventElapsedTime(&t, ev[2 + 2 * k], ev[3 + 2 * k]));
                    sum += t;
                }
                *ms_spmv = (float)sum;
            }
        } catch (...) {
            release();
            throw;
        }
        release();
        // the work buffers and scalars are the step's scratch; the status word may hold what
        // the uncapped loop left: clear it
        SDC_CUDA_TRY(cudaMemsetAsync(&c->st->status, 0, sizeof(int), c->stream));
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
}

sdc_status sdc_set_stationary_state(sdc_ctx* c, double t0, double rtol, int32_t max_iter, int32_t* iters) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(rtol > 0.0 && max_iter > 0, SDC_ERR_ARG, "rtol and max_iter must be positive");
        const size_t bytes = (size_t)c->n * sizeof(double);
        // K T0 = g is the implicit-stage system with zero mass and dtau = 1: a device vector of
        // zeros stands in for m for this one solve
        void* zero = nullptr;
        if (c->alloc) {
            zero = c->alloc(bytes, c->user);
            if (!zero) throw ApiError(SDC_ERR_OOM, "device allocation of the zero mass vector failed");
        } else if (cudaMalloc(&zero, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw ApiError(SDC_ERR_OOM, "cudaMalloc of the zero mass vector failed");
        }
        auto release = [&] {
            cudaStreamSynchronize(c->stream);
            if (c->alloc) c->free_fn(zero, c->user);
            else cudaFree(zero);
        };
        try {
            SDC_CUDA_TRY(cudaMemsetAsync(zero, 0, bytes, c->stream));
            if (!c->temp_set) SDC_CUDA_TRY(cudaMemsetAsync(c->Tn, 0, bytes, c->stream));  // initial guess 0
            // the time of the state, and a clear status for the solve to report into
            StepState* h = c->st_host;
            std::memset(h, 0, sizeof(StepState));
            h->t0 = t0;
            h->dt = c->scheme_set ? c->dt : 1.0;
            SDC_CUDA_TRY(cudaMemcpyAsync(c->st, h, sizeof(StepState), cudaMemcpyHostToDevice, c->stream));
            cudaGraph_t g;
            SDC_CUDA_TRY(cudaGraphCreate(&g, 0));
            std::unique_ptr<CUgraph_st, decltype(&cudaGraphDestroy)> guard(g, &cudaGraphDestroy);
            Chain ch(g);
            CgArgs a = cg_args(c, 1.0, 0, rtol, max_iter);
            a.mass = static_cast<const double*>(zero);
            RhsArgs r{};
            r.mode = RHS_GIVEN;
            r.b_in = c->d_genv;
            r.x0 = c->Tn;
            r.pos = c->C.pos;
            add_solve(c, ch, a, r);
            ch.copy(c->Tn, c->X, bytes);
            cudaGraphExec_t ex;
            SDC_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
            cudaError_t e = cudaGraphLaunch(ex, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            cudaGraphExecDestroy(ex);
            SDC_CUDA_TRY(e);
            int it = 0;
            SDC_CUDA_TRY(cudaMemcpy(&it, &c->st->cg_iters[0], sizeof(int), cudaMemcpyDeviceToHost));
            if (iters) *iters = it;
            c->temp_set = true;
            read_state(c, nullptr);
        } catch (...) {
            release();
            throw;
        }
        release();
    });
}

sdc_status sdc_contact_flux(sdc_ctx* c, const double* T, double t, double* fE) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(T && fE, SDC_ERR_ARG, "null buffer");
        GeomArgs ga{};
        ga.C = c->C;
        ga.E = c->E1;
        ga.slot_pos = nullptr;
        ga.st = c->st;
        ga.t_fixed = t;
        ga.use_fixed = 1;
        ga.n_slots = 1;
        ga.status = &c->st->status;
        const int NI = c->C.n_iface;
        SDC_CUDA_TRY(cudaMemsetAsync(fE, 0, (size_t)c->n * sizeof(double), c->stream));
        k_iface_geom<<<dim3(blocks_for(NI, GEOM_THREADS), 1), GEOM_THREADS, 0, c->stream>>>(ga);
        k_contact_apply<<<blocks_for(NI, 256), 256, 0, c->stream>>>(c->C, c->E1, 0, T, c->Ti1, fE, 0);
        k_contact_apply<<<blocks_for(NI, 256), 256, 0, c->stream>>>(c->C, c->E1, 0, T, c->Ti1, fE, 1);
        SDC_CUDA_TRY(cudaGetLastError());
        read_state(c, nullptr);
    });
}

}  // extern "C"

// ============================================================================ allocation-free heat ledger
//
// sdc_heat_totals_noalloc runs the heat-ledger reduction k_heat with its
// scratch (per-block partial sums, then the arrival counter of the
// last-block combination) in the fixed device array below instead of the
// context's buffers, so the call itself never allocates device memory.
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 32768;
constexpr int64_t NOALLOC_MAX_DOF = (int64_t)NOALLOC_MAX_BLOCKS * RED_BLOCK;      // 8,388,608
constexpr size_t NOALLOC_PARTIAL_BYTES = 2 * (size_t)NOALLOC_MAX_BLOCKS * sizeof(double);  // 512 KiB
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_PARTIAL_BYTES + 256;             // + counter

// Host code must not use this name as an address: the host-side symbol is a
// stand-in. Its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on `device`, looked up once per device
// with that device current (the caller makes it current).
unsigned char* noalloc_scratch(int device) {
    require(device >= 0 && device < NOALLOC_MAX_DEVICES, SDC_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            throw ApiError(SDC_ERR_CUDA, std::string("cudaGetSymbolAddress of the heat-ledger scratch failed: ") +
                                             cudaGetErrorString(e));
        }
        g_noalloc_addr[device] = p;
    }
    return static_cast<unsigned char*>(g_noalloc_addr[device]);
}

// True if p is device memory of GPU `device` (cudaPointerGetAttributes allocates
// nothing). Host, pinned-host and unregistered pointers, and other GPUs' memory, are
// refused before a kernel could write through them.
bool on_device(const void* p, int device) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

// Makes `device` current for the scope and restores the caller's device.
struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int device) {
        SDC_CUDA_TRY(cudaGetDevice(&prev));
        if (prev != device) SDC_CUDA_TRY(cudaSetDevice(device));
    }
    ~CurrentDevice() {
        int now = -1;
        if (cudaGetDevice(&now) == cudaSuccess && now != prev && prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" sdc_status sdc_heat_totals_noalloc(sdc_ctx* c, const double* T_dev, double* heat_dev) {
    return guarded(c, [&] {
        require(c->assembled, SDC_ERR_STATE, "call sdc_assemble first");
        require(T_dev && heat_dev, SDC_ERR_ARG, "null buffer");
        require(c->n <= NOALLOC_MAX_DOF, SDC_ERR_ARG,
                "sdc_heat_totals_noalloc handles at most 8,388,608 DOF (its fixed scratch holds 32,768 "
                "block partials); use sdc_get_heat_totals for larger models");
        require(on_device(T_dev, c->device), SDC_ERR_ARG,
                "T_dev is not device memory of the context's GPU");
        require(on_device(heat_dev, c->device), SDC_ERR_ARG,
                "heat_dev is not device memory of the context's GPU");
        CurrentDevice on(c->device);
        unsigned char* base = noalloc_scratch(c->device);
        double* partials = reinterpret_cast<double*>(base);
        unsigned int* counter = reinterpret_cast<unsigned int*>(base + NOALLOC_PARTIAL_BYTES);
        SDC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), c->stream));
        // one block at least, as the step's own ledger launch: a model without DOFs gets zeros
        k_heat<<<blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK), RED_BLOCK, 0, c->stream>>>(
            c->d_mass, T_dev, c->n, c->n_fix, partials, counter, heat_dev);
        SDC_CUDA_TRY(cudaGetLastError());
    });
}

// ============================================================================ batches

struct sdc_batch {
    int device = 0;
    std::vector<sdc_ctx*> members;
    std::string err;
    // fused group (sdc_batch_set_fused): the members whose inner FP32 CG runs as one launch
    int fused = 0;
    bool group_dirty = true;
    std::vector<sdc_ctx*> group;
    cudaStream_t gstream = nullptr;
    cudaGraph_t ggraph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t gdone = nullptr;
    std::vector<void*> gbufs;       // device buffers of the group graph
};

extern "C" sdc_status sdc_poll(sdc_ctx* c, int* idle) {
    return guarded(c, [&] {
        require(idle != nullptr, SDC_ERR_ARG, "idle is NULL");
        const cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            *idle = 0;
            return;
        }
        SDC_CUDA_TRY(e);
        *idle = 1;
    });
}

namespace {

template <class F>
sdc_status batch_guarded(sdc_batch* b, F&& f) {
    if (!b) return SDC_ERR_ARG;
    try {
        f();
        return SDC_OK;
    } catch (const ApiError& e) {
        b->err = e.what;
        return e.code;
    } catch (const CudaError& e) {
        cudaGetLastError();
        b->err = e.what;
        return e.code == cudaErrorMemoryAllocation ? SDC_ERR_OOM : SDC_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        b->err = "host allocation failed";
        return SDC_ERR_OOM;
    }
}

// a member call failed: carry its message into the batch
void member_check(sdc_ctx* c, sdc_status st, int i) {
    if (st != SDC_OK) throw ApiError(st, "member " + std::to_string(i) + ": " + c->err);
}

// ---------------------------------------------------------------- fused group
//
// The members of a fused group share one CUDA graph per batched macro step. Each member's
// kernels form a chain of that graph as in its own step graph, except its mixed-precision
// implicit solves: there the member's k_mx_init is followed by one group solve, a WHILE
// loop of refinement passes around a WHILE loop of FP32 CG iterations in which each SpMV
// and each update is ONE launch over the concatenated blocks of every member (the
// block-diagonal operator of all members), then one refinement launch. A member's blocks
// use its own arguments, partial sums and scalars, so its arithmetic (block partition and
// summation order included) is that of its own launches and its results are bitwise those
// of the member run alone; a member whose CG stopped returns at once from the later
// launches, and the loops end when the last member stops. Every member's chain waits for
// the group solve before it goes on. Eligible: mixed precision, MRSDC, grids of at most
// MIX_DEFER_MAX_BLOCKS blocks (deferred dots), no diagnostics, graph execution, and the
// same scheme (the same sequence of solves) and matrix form as the group's first member.
bool fusable(const sdc_ctx* c, const sdc_ctx* ref) {
    const bool ok = c->precision == SDC_MIXED_FP32 && c->stepper == SDC_STEPPER_MRSDC && !c->residuals &&
                    !c->true_res && !c->eager &&
                    blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK) <= (unsigned)MIX_DEFER_MAX_BLOCKS;
    if (!ok || !ref) return ok;
    return c->W.kind == ref->W.kind && c->W.M == ref->W.M && c->W.P == ref->W.P && c->W.w == ref->W.w &&
           c->K_sweeps == ref->K_sweeps && c->dt == ref->dt && c->nondeg == ref->nondeg && c->c32 == ref->c32 &&
           c->implied == ref->implied;
}

void group_release(sdc_batch* b) {
    if (b->gstream) cudaStreamSynchronize(b->gstream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->ggraph) cudaGraphDestroy(b->ggraph);
    b->gexec = nullptr;
    b->ggraph = nullptr;
    for (void* p : b->gbufs) cudaFree(p);
    b->gbufs.clear();
    b->group.clear();
    b->group_dirty = true;
}

template <class T>
T* group_upload(sdc_batch* b, const std::vector<T>& v) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw ApiError(SDC_ERR_OOM, "cudaMalloc of a fused-group table failed");
    }
    b->gbufs.push_back(p);
    if (!v.empty()) SDC_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return static_cast<T*>(p);
}

// Member and first-block tables of one fused launch, from each member's block count.
GroupLaunch group_blocks(sdc_batch* b, const std::vector<int>& counts, unsigned& total) {
    std::vector<int> member, first(counts.size() + 1, 0);
    for (size_t m = 0; m < counts.size(); ++m) {
        first[m + 1] = first[m] + counts[m];
        member.insert(member.end(), counts[m], (int)m);
    }
    total = (unsigned)first.back();
    GroupLaunch L{};
    L.member = group_upload(b, member);
    L.first = group_upload(b, first);
    return L;
}

void build_group(sdc_batch* b) {
    group_release(b);
    for (sdc_ctx* c : b->members)
        if (fusable(c, b->group.empty() ? nullptr : b->group[0])) b->group.push_back(c);
    if (b->group.size() < 2) {  // nothing to fuse: every member runs its own graph
        b->group.clear();
        b->group_dirty = false;
        return;
    }
    if (!b->gstream) SDC_CUDA_TRY(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
    if (!b->gdone) SDC_CUDA_TRY(cudaEventCreateWithFlags(&b->gdone, cudaEventDisableTiming));
    const size_t nm = b->group.size();
    GroupState* gs = group_upload(b, std::vector<GroupState>(1, GroupState{0, 0}));
    SDC_CUDA_TRY(cudaGraphCreate(&b->ggraph, 0));
    cudaGraph_t G = b->ggraph;
    std::vector<std::vector<cudaGraphNode_t>> in(nm), out(nm);
    std::vector<std::vector<MixArgs>> args(nm);
    for (size_t i = 0; i < nm; ++i) {
        sdc_ctx* c = b->group[i];
        ensure_ready(c);
        Chain ch(G);
        ch.allow_branches = false;
        std::function<void(Chain&, MixArgs, const RhsArgs&)> hook = [&](Chain& chh, MixArgs a, const RhsArgs& r) {
            a.grp = gs;
            a.h_outer = a.h_inner = 0;
            a.tail_pairs = 0;
            chh.kernel(MK(c, k_mx_init), row_grid(c, MK(c, k_mx_init)), RED_BLOCK, a, r);
            in[i].push_back(chh.last);
            cudaGraphNode_t e;
            SDC_CUDA_TRY(cudaGraphAddEmptyNode(&e, G, nullptr, 0));
            chh.last = e;
            out[i].push_back(e);
            args[i].push_back(a);
        };
        c->solve_hook = &hook;
        try {
            emit_step(c, ch);
        } catch (...) {
            c->solve_hook = nullptr;
            throw;
        }
        c->solve_hook = nullptr;
        require(in[i].size() == in[0].size(), SDC_ERR_STATE, "fused members differ in their solves");
    }
    std::vector<int> n_spmv(nm), n_upd(nm);
    for (size_t i = 0; i < nm; ++i) {
        n_spmv[i] = (int)row_grid(b->group[i], MK32(b->group[i], k_mx_spmv));
        n_upd[i] = (int)b->group[i]->update_grid;
    }
    unsigned t_spmv = 0, t_upd = 0, t_ref = 0;
    GroupArgs g0{};
    g0.gs = gs;
    g0.n_members = (int)nm;
    // beyond what any member's own caps allow (MIX_INNER_MAX iterations, MIX_MAX_REFINE passes)
    g0.launch_cap = 2 * MIX_INNER_MAX + 16;
    g0.pass_cap = MIX_MAX_REFINE + 2;
    g0.spmv = group_blocks(b, n_spmv, t_spmv);
    g0.update = group_blocks(b, n_upd, t_upd);
    g0.refine = group_blocks(b, n_spmv, t_ref);  // the refinement runs one row a thread, like the SpMV
    const int unroll = cg_unroll(b->group[0]);
    for (size_t k = 0; k < in[0].size(); ++k) {
        std::vector<MixArgs> ak(nm);
        for (size_t i = 0; i < nm; ++i) ak[i] = args[i][k];
        GroupArgs g = g0;
        g.args = group_upload(b, ak);
        Chain gc(G);
        for (size_t i = 0; i < nm; ++i) gc.join(in[i][k]);
        cudaGraphConditionalHandle ho, hi;
        SDC_CUDA_TRY(cudaGraphConditionalHandleCreate(&ho, G, 1u, cudaGraphCondAssignDefault));
        g.h_outer = (unsigned long long)ho;
        gc.kernel(k_group_begin, 1u, 32u, g);
        Chain outer(gc.while_node(ho));
        SDC_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, outer.g, 1u, cudaGraphCondAssignDefault));
        g.h_inner = (unsigned long long)hi;
        Chain inner(outer.while_node(hi));
        for (int u = 0; u < unroll; ++u) {
            GroupArgs gu = g;
            gu.tail_pairs = unroll - 1 - u;
            inner.kernel(MK32(b->group[0], k_mx_spmv_g), t_spmv, (unsigned)RED_BLOCK, gu);
            inner.kernel(k_mx_update_g, t_upd, (unsigned)RED_BLOCK, gu);
        }
        outer.kernel(MK32(b->group[0], k_mx_refine_g), t_ref, (unsigned)RED_BLOCK, g);
        gc.kernel(k_group_end, 1u, 32u, g);
        for (size_t i = 0; i < nm; ++i) SDC_CUDA_TRY(cudaGraphAddDependencies(G, &gc.last, &out[i][k], nullptr, 1));
    }
    SDC_CUDA_TRY(cudaGraphInstantiate(&b->gexec, G, 0));
    b->group_dirty = false;
}

}  // namespace

extern "C" sdc_status sdc_batch_create(sdc_batch** out, int device) {
    if (!out) return SDC_ERR_ARG;
    *out = nullptr;
    sdc_batch* b = new (std::nothrow) sdc_batch();
    if (!b) return SDC_ERR_OOM;
    b->device = device;
    *out = b;
    return SDC_OK;
}

extern "C" void sdc_batch_destroy(sdc_batch* b) {
    if (!b) return;
    group_release(b);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->gdone) cudaEventDestroy(b->gdone);
    delete b;
}

extern "C" sdc_status sdc_batch_set_fused(sdc_batch* b, int on) {
    return batch_guarded(b, [&] {
        if (!on) group_release(b);
        b->fused = on ? 1 : 0;
        b->group_dirty = true;
    });
}

extern "C" sdc_status sdc_batch_fused_size(sdc_batch* b, int32_t* n) {
    return batch_guarded(b, [&] {
        require(n != nullptr, SDC_ERR_ARG, "n is NULL");
        if (b->fused && b->group_dirty) build_group(b);
        *n = b->fused ? (int32_t)b->group.size() : 0;
    });
}

extern "C" const char* sdc_batch_last_error(const sdc_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" sdc_status sdc_batch_add(sdc_batch* b, sdc_ctx* c, int32_t* index) {
    return batch_guarded(b, [&] {
        require(c != nullptr, SDC_ERR_ARG, "null context");
        require(c->device == b->device, SDC_ERR_ARG, "the context is on another device");
        require(c->assembled && c->scheme_set && c->temp_set, SDC_ERR_STATE,
                "a member must be assembled, with scheme and temperature set");
        for (sdc_ctx* m : b->members) {
            require(m != c, SDC_ERR_ARG, "the context is already a member");
            require(m->stream != c->stream, SDC_ERR_ARG, "every member needs its own stream");
        }
        b->group_dirty = true;
        b->members.push_back(c);
        c->in_batch += 1;
        c->graph_ready = false;
        if (index) *index = (int32_t)b->members.size() - 1;
    });
}

extern "C" sdc_status sdc_batch_remove(sdc_batch* b, sdc_ctx* c) {
    return batch_guarded(b, [&] {
        auto it = std::find(b->members.begin(), b->members.end(), c);
        require(it != b->members.end(), SDC_ERR_ARG, "not a member");
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (b->fused) group_release(b);
        b->members.erase(it);
        c->in_batch -= 1;
        c->graph_ready = false;
    });
}

extern "C" sdc_status sdc_batch_size(const sdc_batch* cb, int32_t* n) {
    sdc_batch* b = const_cast<sdc_batch*>(cb);
    return batch_guarded(b, [&] {
        require(n != nullptr, SDC_ERR_ARG, "n is NULL");
        *n = (int32_t)b->members.size();
    });
}

extern "C" sdc_status sdc_batch_step(sdc_batch* b, const int64_t* n_steps, int wait) {
    return batch_guarded(b, [&] {
        const size_t nm = b->members.size();
        int64_t most = 0;
        for (size_t i = 0; i < nm; ++i) {
            const int64_t k = n_steps ? n_steps[i] : 1;
            require(k >= 0, SDC_ERR_ARG, "negative step count");
            most = std::max(most, k);
        }
        // fused group: rebuilt when the membership or a member's options changed
        if (b->fused) {
            bool dirty = b->group_dirty;
            for (sdc_ctx* c : b->members) dirty = dirty || !c->graph_ready || !c->buffers_ready;
            if (dirty) build_group(b);
        }
        auto in_group = [&](sdc_ctx* c) {
            return b->fused && std::find(b->group.begin(), b->group.end(), c) != b->group.end();
        };
        int64_t group_steps = -1;
        for (size_t i = 0; i < nm; ++i) {  // graphs and buffers first, outside the launch sweep
            sdc_ctx* c = b->members[i];
            const int64_t k = n_steps ? n_steps[i] : 1;
            if (in_group(c)) {
                require(group_steps < 0 || group_steps == k, SDC_ERR_ARG,
                        "the fused members of a batch step together: give them equal step counts");
                group_steps = k;
            }
            if (k > 0) member_check(c, guarded(c, [&] { ensure_ready(c); }), (int)i);
        }
        if (group_steps > 0) {  // the group's graph runs after the work already on the members' streams
            for (sdc_ctx* c : b->group) {
                SDC_CUDA_TRY(cudaEventRecord(b->gdone, c->stream));
                SDC_CUDA_TRY(cudaStreamWaitEvent(b->gstream, b->gdone, 0));
            }
        }
        for (int64_t s = 0; s < most; ++s) {
            if (s < group_steps) SDC_CUDA_TRY(cudaGraphLaunch(b->gexec, b->gstream));
            for (size_t i = 0; i < nm; ++i) {
                sdc_ctx* c = b->members[i];
                if (in_group(c)) continue;
                if (s < (n_steps ? n_steps[i] : 1)) member_check(c, guarded(c, [&] { launch_step(c); }), (int)i);
            }
        }
        if (group_steps > 0) {  // and later work on a member's stream runs after the group's steps
            SDC_CUDA_TRY(cudaEventRecord(b->gdone, b->gstream));
            for (sdc_ctx* c : b->group) SDC_CUDA_TRY(cudaStreamWaitEvent(c->stream, b->gdone, 0));
        }
        if (wait)
            for (size_t i = 0; i < nm; ++i) member_check(b->members[i], sdc_synchronize(b->members[i]), (int)i);
    });
}

extern "C" sdc_status sdc_batch_synchronize(sdc_batch* b) {
    return batch_guarded(b, [&] {
        for (size_t i = 0; i < b->members.size(); ++i)
            member_check(b->members[i], sdc_synchronize(b->members[i]), (int)i);
    });
}


// ============================================================================ autotuner
//
// sdc_autotune picks the launch options of a context's macro-step graph from timed trial
// steps: (SpMV, update) pairs per CG loop body, the blocks a SM of the deferred FP32 update,
// the cap on the contact loop's cluster, the placement of its replicas, and graph side
// branches. Every option leaves results bitwise unchanged (fixed-order reductions whose
// order does not depend on them), so only time is compared. Each candidate is timed on the
// same macro steps from the same saved state (T(t_n) and the step counters), by coordinate
// descent from the context's current options; a candidate is taken when it is at least 1 %
// faster. Picks are cached per process by the shape of the problem (device, sizes, contact
// DOFs, precision, stepper, scheme), so contexts of equal shape (the members of a batch,
// the slots of the serving loop) are tuned once.
namespace {

struct TuneOpts {
    int unroll, update_bps, cluster_cap, global, branches;
};

struct TuneKey {
    int device, precision, stepper, nodes, M, P, K;
    int64_t n, nnz, n_iface;
    bool operator<(const TuneKey& o) const {
        return std::tie(device, precision, stepper, nodes, M, P, K, n, nnz, n_iface) <
               std::tie(o.device, o.precision, o.stepper, o.nodes, o.M, o.P, o.K, o.n, o.nnz, o.n_iface);
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneOpts> g_tune_cache;

TuneKey tune_key(const sdc_ctx* c) {
    return {c->device, c->precision, c->stepper, c->W.kind, c->W.M, c->W.P, c->K_sweeps,
            c->n, c->nnz, (int64_t)c->C.n_iface};
}

TuneOpts current_opts(sdc_ctx* c) {
    int bps = c->update_bps;
    if (bps == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mx_update, RED_BLOCK, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        bps = std::max(per_sm, 1);
    }
    return {cg_unroll(c), bps, c->max_cluster, c->force_global, c->branches};
}

void apply_opts(sdc_ctx* c, const TuneOpts& o) {
    if (o.cluster_cap != c->max_cluster || o.global != c->force_global) c->buffers_ready = false;
    c->cg_unroll = o.unroll;
    c->update_bps = o.update_bps;
    c->max_cluster = o.cluster_cap;
    c->force_global = o.global;
    c->branches = o.branches;
    set_update_grid(c);
    c->graph_ready = false;
}

// Device state a trial step changes, saved once and restored before every timed trial.
struct TuneSnapshot {
    sdc_ctx* c;
    void* T = nullptr;
    StepState st{};
    explicit TuneSnapshot(sdc_ctx* cc) : c(cc) {
        const size_t bytes = (size_t)c->n * sizeof(double);
        if (c->alloc) T = c->alloc(bytes, c->user);
        else if (cudaMalloc(&T, bytes) != cudaSuccess) {
            cudaGetLastError();
            T = nullptr;
        }
        if (!T) throw ApiError(SDC_ERR_OOM, "device allocation of the autotuner's state copy failed");
        SDC_CUDA_TRY(cudaMemcpyAsync(T, c->Tn, bytes, cudaMemcpyDeviceToDevice, c->stream));
        SDC_CUDA_TRY(cudaMemcpyAsync(&st, c->st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream));
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    void restore() {
        SDC_CUDA_TRY(cudaMemcpyAsync(c->Tn, T, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        SDC_CUDA_TRY(cudaMemcpyAsync(c->st, &st, sizeof(StepState), cudaMemcpyHostToDevice, c->stream));
        SDC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    ~TuneSnapshot() {
        if (!T) return;
        cudaStreamSynchronize(c->stream);
        if (c->alloc) c->free_fn(T, c->user);
        else cudaFree(T);
    }
};

// ms per macro step of the context's current options: one untimed step (graph build and
// first launch), then the best of two runs of `steps` steps, each from the saved state.
double time_opts(sdc_ctx* c, TuneSnapshot& snap, int steps) {
    ensure_ready(c);
    snap.restore();
    launch_step(c);
    read_state(c, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SDC_CUDA_TRY(cudaEventCreate(&e0));
    SDC_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e300;
    try {
        for (int rep = 0; rep < 2; ++rep) {
            snap.restore();
            SDC_CUDA_TRY(cudaEventRecord(e0, c->stream));
            for (int s = 0; s < steps; ++s) launch_step(c);
            SDC_CUDA_TRY(cudaEventRecord(e1, c->stream));
            SDC_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            SDC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            read_state(c, nullptr);
            best = std::min(best, (double)ms / steps);
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" sdc_status sdc_autotune(sdc_ctx* c, int32_t trial_steps, sdc_tune_report* rep) {
    return guarded(c, [&] {
        require(trial_steps >= 0 && trial_steps <= 64, SDC_ERR_ARG, "trial_steps out of range [0, 64]");
        require(!c->eager, SDC_ERR_STATE, "autotuning times graph execution: switch eager execution off");
        ensure_ready(c);
        const int steps = trial_steps ? trial_steps : 3;
        const TuneKey key = tune_key(c);
        sdc_tune_report out{};
        out.ms_default = out.ms_tuned = -1.0;
        bool cached = false;
        TuneOpts picked{};
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                picked = it->second;
                cached = true;
            }
        }
        if (cached) {
            apply_opts(c, picked);
            ensure_ready(c);
        } else {
            TuneSnapshot snap(c);
            TuneOpts best = current_opts(c);
            apply_opts(c, best);
            double best_ms = time_opts(c, snap, steps);
            out.ms_default = best_ms;
            int trials = 1;
            // a candidate the device cannot run (e.g. a contact cluster too small for every
            // loop form) is skipped; the context then takes the best options again
            auto consider = [&](TuneOpts o) {
                double ms = 0.0;
                try {
                    apply_opts(c, o);
                    ms = time_opts(c, snap, steps);
                } catch (const ApiError& e) {
                    if (e.code != SDC_ERR_CUDA && e.code != SDC_ERR_ARG) throw;
                    cudaGetLastError();
                    apply_opts(c, best);
                    ensure_ready(c);
                    ++out.skipped;
                    return;
                }
                ++trials;
                if (ms < 0.99 * best_ms) {
                    best = o;
                    best_ms = ms;
                }
            };
            const bool small_grid = blocks_for(std::max<int64_t>(c->n, 1), RED_BLOCK) <= (unsigned)MIX_DEFER_MAX_BLOCKS;
            for (int u : small_grid ? std::vector<int>{1, 2, 3, 4, 6} : std::vector<int>{1, 2})
                if (u != best.unroll) consider({u, best.update_bps, best.cluster_cap, best.global, best.branches});
            if (c->precision == SDC_MIXED_FP32 && small_grid) {
                const int top = best.update_bps;
                for (int b = 2; b < top; ++b) consider({best.unroll, b, best.cluster_cap, best.global, best.branches});
            }
            // smaller clusters than the automatic size (the cap never enlarges it); a grid-wide
            // loop is tried against the largest cluster instead
            const int auto_cs = c->iface_grid ? 2 * IFACE_MAX_CLUSTER : c->iface_cluster;
            for (int cs = auto_cs / 2; cs >= 1 && cs >= auto_cs / 4; cs /= 2)
                consider({best.unroll, best.update_bps, cs, best.global, best.branches});
            // replica placement, from the layout the best options give
            apply_opts(c, best);
            ensure_ready(c);
            const bool best_global = c->iface_global, best_stage = c->iface_stage, best_grid = c->iface_grid;
            if (!best_global) {
                consider({best.unroll, best.update_bps, best.cluster_cap, 1, best.branches});
                consider({best.unroll, best.update_bps, best.cluster_cap, 2, best.branches});
            } else if (best_stage) {
                consider({best.unroll, best.update_bps, best.cluster_cap, 2, best.branches});
            }
            if (!best_grid) consider({best.unroll, best.update_bps, 0, 3, best.branches});
            if (!c->in_batch) consider({best.unroll, best.update_bps, best.cluster_cap, best.global, 1 - best.branches});
            apply_opts(c, best);
            ensure_ready(c);
            snap.restore();
            out.ms_tuned = best_ms;
            out.trials = trials;
            picked = best;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[key] = best;
        }
        out.cg_unroll = picked.unroll;
        out.update_blocks_per_sm = picked.update_bps;
        out.contact_cluster_cap = picked.cluster_cap;
        out.contact_cluster = c->iface_cluster;
        out.contact_global = c->iface_grid ? 3 : c->iface_global ? (c->iface_stage ? 1 : 2) : 0;
        out.graph_branches = picked.branches;
        out.cached = cached ? 1 : 0;
        if (rep) *rep = out;
    });
}
