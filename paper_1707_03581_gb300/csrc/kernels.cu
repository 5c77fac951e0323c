// CUDA kernels of the IMEX multi-rate SDC step (sm_103a).
//
// Memory-bound work (sliced-ELL SpMV, CG vector updates, right-hand sides)
// runs one row per thread with the slice layout giving coalesced loads of
// values and column ids; reductions finish in the last block to arrive
// (fixed-order combination, no floating-point atomics, so results are
// reproducible run to run). The contact substep loop runs on one
// thread-block cluster synchronised with hardware cluster barriers.
#include <cooperative_groups.h>
#include <type_traits>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace sdc {

// ------------------------------------------------------------------ helpers

// A step's status word: the first error reported stays (a give-up of a bounded wait is not
// overwritten by the non-convergence that its garbage causes later in the step).
__device__ __forceinline__ void report_status(int* status, sdc_status code) { atomicCAS(status, 0, (int)code); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// sum_k K[row, k] x[k] over the sliced-ELL row (padding entries carry 0).
// Entries are taken CH at a time: the CH value and column loads of a chunk
// are all issued before its CH gathers of x, so a row costs ceil(w / CH)
// dependent memory round trips instead of w. Summation stays in entry order.
// The thread of the slice's first row first asks for the slice's values and columns (two
// contiguous ranges: 32 w entries, so 16-byte aligned) to be brought into L2 with one bulk
// prefetch each, so that only the first chunk waits for HBM: measured on the 5.75M-row FP32
// matrix (27-point rows, 16-bit columns, 8 blocks of 256 a SM), 194 us without it and 163 us
// with it and 6 entries a chunk, 0.91 of measured HBM.
// C32: the matrix's column form (a kernel template parameter, so that each kernel has the
// registers of one form): 32-bit columns, or 16-bit offsets from each slice's base.
template <bool C32, int CH, typename V, typename X>
__device__ __forceinline__ V ell_row_t(const EllDev& A, const V* __restrict__ val, int64_t row,
                                       const X* __restrict__ x) {
    const int64_t s = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t b = A.slice_ptr[s], e = A.slice_ptr[s + 1];
    if (lane == 0) {
        const unsigned vb = (unsigned)((e - b) * sizeof(V));
        const unsigned cbytes = (unsigned)((e - b) * (C32 ? sizeof(int32_t) : sizeof(uint16_t)));
        const void* cp = C32 ? (const void*)(A.col + b) : (const void*)(A.off + b);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(val + b), "r"(vb) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(cp), "r"(cbytes) : "memory");
    }
    const int32_t cb = C32 ? 0 : __ldg(A.base + s);
    V acc = V(0);
    for (int64_t k0 = b + lane; k0 < e; k0 += (int64_t)CH * SLICE) {
        V v[CH];
        int64_t c[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int64_t k = k0 + (int64_t)j * SLICE;
            const bool in = k < e;
            v[j] = in ? __ldg(val + k) : V(0);
            if constexpr (C32) c[j] = in ? (int64_t)__ldg(A.col + k) : 0;
            else c[j] = in ? (int64_t)(cb + (int32_t)__ldg(A.off + k)) : 0;
        }
        X xv[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) xv[j] = __ldg(x + c[j]);
#pragma unroll
        for (int j = 0; j < CH; ++j) acc = fma(v[j], (V)xv[j], acc);
    }
    return acc;
}

template <bool C32>
__device__ __forceinline__ double ell_row(const EllDev& A, int64_t row, const double* __restrict__ x) {
    return ell_row_t<C32, 4, double, double>(A, A.val, row, x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-reduce NQ values, publish per-block partials, and let the last block
// to finish combine them in a fixed order into out[0..NQ). The warp stage
// runs in the type of v (FP32 for the FP32 kernels: GB300's FP64 pipe is
// narrow, and a warp butterfly costs five adds per value and lane); block and
// grid stages run in FP64. Returns true in every thread of that last block,
// after out[] is written.
template <int NQ, bool MAX, typename W>
__device__ bool reduce_last(W (&v)[NQ], double* partials, unsigned int* counter, double* out) {
    __shared__ double sh[NQ][32];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if constexpr (sizeof(W) == sizeof(float)) {
        // FP32 butterfly in every warp, then FP64 over the warp sums
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = MAX ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh[q][warp] = (double)v[q];
        __syncthreads();
        if (warp == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double t = lane < nw ? sh[q][lane] : (MAX ? -1.0 : 0.0);
                sh[q][lane] = MAX ? warp_max(t) : warp_sum(t);
            }
    } else {
        // FP64: the block's values go to shared memory as columns of 32; warp 0 alone sums the
        // columns, then one butterfly (about a third of the FP64 warp instructions of a
        // butterfly in every warp)
        __shared__ double colv[NQ][RED_BLOCK];
#pragma unroll
        for (int q = 0; q < NQ; ++q) colv[q][threadIdx.x] = v[q];
        __syncthreads();
        if (warp == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double t = colv[q][lane];
                for (int w = 1; w < nw; ++w) t = MAX ? fmax(t, colv[q][lane + 32 * w]) : t + colv[q][lane + 32 * w];
                sh[q][lane] = MAX ? warp_max(t) : warp_sum(t);
            }
    }
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (lane == 0) partials[(size_t)q * gridDim.x + blockIdx.x] = sh[q][0];
        if (lane == 0) {
            __threadfence();
            const unsigned int prev = atomicAdd(counter, 1u);
            am_last = (prev == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double dv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double t = MAX ? -1.0 : 0.0;
        for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
            const double p = __ldcg(partials + (size_t)q * gridDim.x + i);
            t = MAX ? fmax(t, p) : t + p;
        }
        dv[q] = MAX ? warp_max(t) : warp_sum(t);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sh[q][warp] = dv[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = MAX ? -1.0 : 0.0;
            for (int w = 0; w < nw; ++w) t = MAX ? fmax(t, sh[q][w]) : t + sh[q][w];
            out[q] = t;
        }
        *counter = 0u;
    }
    __syncthreads();
    return true;
}

// FP32 row of the implied-column layout (A.stab set): entry k of the row is column
// row + stoff[t + k] of the slice's table t, so only values stream from memory (4 bytes an
// entry) and the table, one per slice shape, comes from L1 with one broadcast load per entry
// for the warp. A slice flagged by ~t clamps its columns to [0, n); the clamped entries hold 0.
// The entries run in increasing column, so the products and their order are those of the
// offsets form (the zeros of absent neighbours add nothing).
template <int CH>
__device__ __forceinline__ float ell_row_implied(const EllDev& A, int64_t row, const float* __restrict__ x) {
    const int64_t s = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t b = A.slice_ptr32[s], e = A.slice_ptr32[s + 1];
    if (lane == 0) {
        const unsigned vb = (unsigned)((e - b) * sizeof(float));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A.val32 + b), "r"(vb) : "memory");
    }
    int32_t q = __ldg(A.stab + s);  // table position of the chunk's first entry
    const bool clamp = q < 0;
    if (clamp) q = ~q;
    const int32_t r = (int32_t)row;
    float acc = 0.0f;
    for (int64_t k0 = b + lane; k0 < e; k0 += (int64_t)CH * SLICE, q += CH) {
        float v[CH];
        int32_t c[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int64_t k = k0 + (int64_t)j * SLICE;
            const bool in = k < e;  // entry (k - b) / 32 of a table of (e - b) / 32 entries
            v[j] = in ? __ldg(A.val32 + k) : 0.0f;
            int32_t cc = in ? r + __ldg(A.stoff + (q + j)) : r;
            if (clamp) cc = min(max(cc, 0), (int32_t)A.n - 1);
            c[j] = cc;
        }
        float xv[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) xv[j] = __ldg(x + c[j]);
#pragma unroll
        for (int j = 0; j < CH; ++j) acc = fmaf(v[j], xv[j], acc);
    }
    return acc;
}

// FP32 row of the sliced ELL: sum_k K32[row, k] x[k], CH entries a chunk (6; the fused batch
// group's kernels, which hold their member's tables too, take 4 to keep within 32 registers).
// F is the FP32 copy's form: 0 = 16-bit offsets, 1 = 32-bit columns, 2 = implied columns.
template <int F, int CH = 6>
__device__ __forceinline__ float ell_row32(const EllDev& A, int64_t row, const float* __restrict__ x) {
    if constexpr (F == 2) return ell_row_implied<CH>(A, row, x);
    else return ell_row_t<F == 1, CH, float, float>(A, A.val32, row, x);
}

// Two-level form of reduce_last for the CG kernels. Block totals go to
// partials; the last block of each group of RED_GROUP blocks (a per-group
// arrival counter) sums its group with one warp, two loads per lane, into
// gpartials; the last group to finish sums the group totals with the whole
// block. Both combinations read their inputs with loads issued together, so
// the tail of the kernel is two short memory round trips, not a serial walk
// over every block's partial. Fixed order throughout.
// counters[0] counts finished groups, counters[1 + g] the blocks of group g.
constexpr int RED_GROUP = 64;

template <int NQ, typename W>
__device__ bool reduce_last2_at(W (&v)[NQ], double* partials, double* gpartials, unsigned int* counters, double* out,
                                unsigned int blk, unsigned int nblk);

template <int NQ, typename W>
__device__ bool reduce_last2(W (&v)[NQ], double* partials, double* gpartials, unsigned int* counters, double* out) {
    return reduce_last2_at<NQ, W>(v, partials, gpartials, counters, out, blockIdx.x, gridDim.x);
}

// The same with the block's index and the grid size given: a fused launch over several
// machines passes each machine's own block index and grid, so that every machine keeps the
// partition and summation order of its own launch.
template <int NQ, typename W>
__device__ bool reduce_last2_at(W (&v)[NQ], double* partials, double* gpartials, unsigned int* counters, double* out,
                                unsigned int blk, unsigned int nblk) {
    __shared__ double sh[NQ][32];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if constexpr (sizeof(W) == sizeof(float)) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh[q][warp] = (double)v[q];
        __syncthreads();
        if (warp == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double t = lane < nw ? sh[q][lane] : 0.0;
                sh[q][lane] = warp_sum(t);
            }
    } else {
        __shared__ double colv[NQ][RED_BLOCK];
#pragma unroll
        for (int q = 0; q < NQ; ++q) colv[q][threadIdx.x] = v[q];
        __syncthreads();
        if (warp == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double t = colv[q][lane];
                for (int w = 1; w < nw; ++w) t += colv[q][lane + 32 * w];
                sh[q][lane] = warp_sum(t);
            }
    }
    const unsigned int g = blk / RED_GROUP;
    const unsigned int ng = (nblk + RED_GROUP - 1) / RED_GROUP;
    const unsigned int gsize = min((unsigned int)RED_GROUP, nblk - g * RED_GROUP);
    if (warp == 0 && lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) partials[(size_t)q * nblk + blk] = sh[q][0];
        __threadfence();
        am_last = atomicAdd(&counters[1 + g], 1u) == gsize - 1;
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double pv[RED_GROUP / 32];
#pragma unroll
            for (int c = 0; c < RED_GROUP / 32; ++c) {
                const unsigned int k = lane + 32 * c;
                pv[c] = k < gsize ? __ldcg(partials + (size_t)q * nblk + g * RED_GROUP + k) : 0.0;
            }
            double t = 0.0;
#pragma unroll
            for (int c = 0; c < RED_GROUP / 32; ++c) t += pv[c];
            t = warp_sum(t);
            if (lane == 0) gpartials[(size_t)q * ng + g] = t;
        }
        if (lane == 0) {
            counters[1 + g] = 0u;
            __threadfence();
            am_last = atomicAdd(&counters[0], 1u) == ng - 1;
        }
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    constexpr int G = 4;
    double dv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) dv[q] = 0.0;
    for (unsigned int base = threadIdx.x; base < ng; base += G * blockDim.x) {
        double pv[NQ][G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            const unsigned int i = base + c * blockDim.x;
#pragma unroll
            for (int q = 0; q < NQ; ++q) pv[q][c] = i < ng ? __ldcg(gpartials + (size_t)q * ng + i) : 0.0;
        }
#pragma unroll
        for (int c = 0; c < G; ++c)
#pragma unroll
            for (int q = 0; q < NQ; ++q) dv[q] += pv[q][c];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) dv[q] = warp_sum(dv[q]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sh[q][warp] = dv[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[q][w];
            out[q] = t;
        }
        counters[0] = 0u;
    }
    __syncthreads();
    return true;
}

// ------------------------------------------------------------------ operator

// y = m .* x + dtau K x
template <bool C32>
__global__ void k_apply_operator(EllDev A, const double* __restrict__ mass, double dtau,
                                 const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.n) {
        y[i] = fma(dtau, ell_row<C32>(A, i, x), mass[i] * x[i]);
    }
}

// F = -K T + g   (f^I(T) + g of Eq. ivp)
template <bool C32>
__global__ void k_fi(EllDev A, const double* __restrict__ g, const double* __restrict__ T, double* __restrict__ F,
                     int* step_counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (step_counts && i == 0) *step_counts = 0;  // step start: kernels launched in the CG loops
    if (i < A.n) {
        F[i] = g[i] - ell_row<C32>(A, i, T);
    }
}

// ------------------------------------------------------------------ Jacobi-PCG

// L_E u on row i for fully implicit Euler: the linear part of the contact term,
// f^E(u, t) = cst + L_E u, from the step's FP64 coupling rows at one slot
// (indices are contact DOFs); 0 off the contact. The FP64 rows are used in both
// precisions: L_E is symmetric, so the operator stays SPD.
__device__ __forceinline__ double ie_contact(const IeOp& o, int64_t i, const double* u) {
    const int pa = o.pos[i];
    if (pa < 0) return 0.0;
    const size_t so = (size_t)o.slot * o.NI + pa;
    const int n = o.E.cnt[so];
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
        const size_t off = ((size_t)o.slot * MAXE + k) * o.NI + pa;
        acc = fma(o.E.coef[off], u[o.dof[o.E.idx[off]]], acc);
    }
    return acc;
}

// Right-hand side of the implicit stage (Algorithm 1: m T_{m-1} + dtau g;
// Algorithm 2: m T^{k+1}_{m-1} - dtau f^I(T^k_m) + I_{m-1}^m), the initial
// residual r = b - (m x0 + dtau K x0), u = D r, and the stop test.
// IE: the operator is m + dtau (K - L_E(t_{n+1})) (contact coupling in the matrix).
template <bool C32, bool IE>
__device__ __forceinline__ void cg_init_impl(const CgArgs& a, const RhsArgs& r) {
    double v[2] = {0.0, 0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
            const double m = a.mass[i];
            double b;
            if (r.mode == RHS_GIVEN) {
                b = r.b_in[i];
            } else if (r.mode == RHS_PRED) {
                b = m * r.Tprev[i] + a.dtau * r.g[i];
                if (r.ihat) {  // contact rows: dtau f^E(T_{m-1}, tau_{m-1}) (single-rate SDC) or
                               // dt f^E(0, t_{n+1}) (implicit Euler)
                    const int pa = r.pos[i];
                    if (pa >= 0) b += r.ihat[pa];
                }
            } else {
                double I = 0.0;
                for (int j = 0; j < r.nFI; ++j) I = fma(r.Sdt[j], r.FI[j][i], I);
                const int pa = r.pos[i];
                if (pa >= 0) I += r.ihat[pa];
                b = m * r.Tprev[i] - a.dtau * (r.FIm[i] - r.g[i]) + I;
            }
            const double x0 = r.x0[i];
            double Kx0 = r.Fx0 ? r.g[i] - r.Fx0[i] : ell_row<C32>(a.A, i, r.x0);
            if constexpr (IE) Kx0 -= ie_contact(a.ie, i, r.x0);
            const double Ax = fma(a.dtau, Kx0, m * x0);
            const double res = b - Ax;
            const double d = 1.0 / (m + a.dtau * a.diagK[i]);
            a.X[i] = x0;
            a.R[i] = res;
            a.D[i] = d;
            a.U[i] = res * d;
            v[0] += b * b;
            v[1] += res * res;
    }
    double out[2];
    if (reduce_last2<2>(v, a.partials, a.gpartials, a.counter, out) && threadIdx.x == 0) {
        CgState* s = a.cg;
        s->bb = out[0];
        s->rr = out[1];
        s->iter = 0;
        s->runs = 0;
        s->beta = 0.0;
        *a.iters_out = 0;
        const bool conv = out[1] <= a.rtol2 * out[0];
        s->done = conv ? 1 : 0;
        if (conv && a.handle) cudaGraphSetConditional((cudaGraphConditionalHandle)a.handle, 0u);
    }
}

template <bool C32>
__global__ void k_cg_init(CgArgs a, RhsArgs r) { cg_init_impl<C32, false>(a, r); }
template <bool C32>
__global__ void k_ie_init(CgArgs a, RhsArgs r) { cg_init_impl<C32, true>(a, r); }

// w = m u + dtau K u (IE: m u + dtau (K - L_E) u); gamma = (r, u), delta = (w, u),
// rr = (r, r). The last block tests ||r|| <= rtol ||b|| (stop) or sets the step
// lengths:
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev).
template <bool C32, bool IE>
__device__ __forceinline__ void cg_spmv_impl(const CgArgs& a) {
    if (a.cg->done) return;  // an iteration queued after convergence (host-driven loop)
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
            const double u = a.U[i];
            double Ku = ell_row<C32>(a.A, i, a.U);
            if constexpr (IE) Ku -= ie_contact(a.ie, i, a.U);
            const double w = fma(a.dtau, Ku, a.mass[i] * u);
            const double res = a.R[i];
            a.W[i] = w;
            v[0] += res * u;
            v[1] += w * u;
            v[2] += res * res;
    }
    double out[3];
    if (reduce_last2<3>(v, a.partials, a.gpartials, a.counter, out) && threadIdx.x == 0) {
        CgState* s = a.cg;
        s->runs += 1;
        *a.loop_kernels += 2;
        const double gamma = out[0], delta = out[1];
        s->rr = out[2];
        const bool conv = out[2] <= a.rtol2 * s->bb;
        if (conv || s->iter >= a.max_iter) {
            *a.loop_kernels += 2 * a.tail_pairs;  // the rest of the loop body runs and returns
            s->done = 1;
            if (!conv) report_status(a.status, SDC_ERR_NOT_CONVERGED);
            if (a.handle) cudaGraphSetConditional((cudaGraphConditionalHandle)a.handle, 0u);
            return;
        }
        if (s->iter == 0) {
            s->beta = 0.0;
            s->alpha = gamma / delta;
        } else {
            const double beta = gamma / s->gamma;
            s->beta = beta;
            s->alpha = gamma / (delta - beta * gamma / s->alpha);
        }
        s->gamma = gamma;
        s->delta = delta;
        s->iter += 1;
        *a.iters_out = s->iter;
    }
}

template <bool C32>
__global__ void k_cg_spmv(CgArgs a) { cg_spmv_impl<C32, false>(a); }
template <bool C32>
__global__ void k_ie_spmv(CgArgs a) { cg_spmv_impl<C32, true>(a); }

// p = u + beta p; s = w + beta s; x += alpha p; r -= alpha s; u = D r
__global__ void k_cg_update(CgArgs a) {
    if (a.cg->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const double alpha = a.cg->alpha, beta = a.cg->beta;
        const bool first = a.cg->iter == 1;
        const double u = a.U[i], w = a.W[i];
        const double p = first ? u : fma(beta, a.P[i], u);
        const double sp = first ? w : fma(beta, a.S[i], w);
        a.P[i] = p;
        a.S[i] = sp;
        a.X[i] = fma(alpha, p, a.X[i]);
        const double res = fma(-alpha, sp, a.R[i]);
        a.R[i] = res;
        a.U[i] = res * a.D[i];
    }
}

// ------------------------------------------------------------------ mixed precision (iterative refinement)

// Start of one refinement pass, by the kernel that formed its FP64 residual
// r (k_mx_init, k_mx_refine): r32 = r and u = D r32 on every row, and here, in
// that kernel's last block, the inner state. The inner target is the larger of
// a fixed FP32 reduction and what the outer test still needs (with a margin for
// the FP32 recurrence), so a pass stops as soon as one more FP64 residual can
// meet ||b - A x|| <= rtol ||b||. The pass's first update sets d (d = alpha p,
// or 0 when the pass stops before it).
__device__ __forceinline__ void mx_begin_pass(const MixArgs& a, double rr) {
    CgState* s = a.cg;
    s->bb = fmax(a.inner_rtol2 * rr, 0.1 * a.rtol2 * a.ms->bb);
    s->rr = rr;
    s->beta = 0.0;
    s->iter = 0;
    s->runs = 0;
    s->done = rr > 0.0 ? 0 : 1;
    s->pending = 0;
    // the inner loop's condition starts at 1 with each step's graph launch; the
    // refinement (in the same graph as that loop) sets it again for each later pass
    if (a.h_inner) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_inner, 1u);
    if (a.grp && !s->done) atomicAdd(&a.grp->inner_active, 1);  // the group's refinement sets the condition
}

// A CG-loop SpMV that finds its solve done on entry. If no kernel of this pass
// has run (the pass had nothing to solve), the first one counts the loop body
// and stops the loop (whose condition is 1 at the start of every pass).
__device__ __forceinline__ void mx_done_on_entry(const MixArgs& a) {
    CgState* s = a.cg;
    if (blockIdx.x == 0 && threadIdx.x == 0 && s->runs == 0) {
        s->runs = -1;
        *a.loop_kernels += a.pair_kernels * (1 + a.tail_pairs);
        if (a.h_inner) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_inner, 0u);
    }
}

// FP64: b of the implicit stage (as k_cg_init), x = x0, r = b - A x0, and
// the outer stop test; FP32 inverse diagonal for the inner solves.
template <bool C32>
__global__ void k_mx_init(MixArgs a, RhsArgs r) {
    double v[2] = {0.0, 0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
            const double m = a.mass[i];
            double b;
            if (r.mode == RHS_GIVEN) {
                b = r.b_in[i];
            } else if (r.mode == RHS_PRED) {
                b = m * r.Tprev[i] + a.dtau * r.g[i];
                if (r.ihat) {  // contact rows: dtau f^E(T_{m-1}, tau_{m-1}) (single-rate SDC) or
                               // dt f^E(0, t_{n+1}) (implicit Euler)
                    const int pa = r.pos[i];
                    if (pa >= 0) b += r.ihat[pa];
                }
            } else {
                double I = 0.0;
                for (int j = 0; j < r.nFI; ++j) I = fma(r.Sdt[j], r.FI[j][i], I);
                const int pa = r.pos[i];
                if (pa >= 0) I += r.ihat[pa];
                b = m * r.Tprev[i] - a.dtau * (r.FIm[i] - r.g[i]) + I;
            }
            const double x0 = r.x0[i];
            const double Kx0 = r.Fx0 ? r.g[i] - r.Fx0[i] : ell_row<C32>(a.A, i, r.x0);
            const double res = b - fma(a.dtau, Kx0, m * x0);
            a.B[i] = b;
            a.X[i] = x0;
            a.R[i] = res;
            a.Dsum[i] = 0.0f;
            const float dinv = 1.0f / (float)(m + a.dtau * a.diagK[i]);
            a.Dinv[i] = dinv;
            a.Rl[i] = (float)res;  // the first pass's FP32 residual and u
            a.Ul[i] = (float)res * dinv;
            v[0] += b * b;
            v[1] += res * res;
    }
    double out[2];
    if (reduce_last2<2>(v, a.partials, a.gpartials, a.counter, out) && threadIdx.x == 0) {
        MixState* s = a.ms;
        s->bb = out[0];
        s->rr = out[1];
        s->passes = 0;
        *a.iters_out = 0;
        *a.refine_out = 0;
        const bool conv = out[1] <= a.rtol2 * out[0];
        s->done = conv ? 1 : 0;
        if (conv) a.cg->done = 1;  // no inner pass: a fused group's loops skip this member
        if (conv && a.h_outer) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer, 0u);
        if (!conv) {
            if (a.grp) atomicAdd(&a.grp->outer_active, 1);
            mx_begin_pass(a, out[1]);
        }
    }
}

// Sums of FP32 values over a block, fixed order (warp butterflies, then warp 0
// over the warp totals); thread 0 writes them to partials[q * gridDim.x + block].
template <int NQ>
__device__ __forceinline__ void block_partials_f32(float (&v)[NQ], float* partials, unsigned int blk, unsigned int nblk) {
    __shared__ float sh[NQ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v[q] = warp_sum(v[q]);
        if (lane == 0) sh[q][warp] = v[q];
    }
    __syncthreads();
    if (warp == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float t = warp_sum(lane < nw ? sh[q][lane] : 0.0f);
            if (lane == 0) partials[(size_t)q * nblk + blk] = t;
        }
}

// Totals of G block partials partials[q * G + b] (written by the previous
// launch; read through L1, so that the blocks on one SM share the lines that
// every block reads: 4.6 against 5.8 us an update at 313k rows in a probe), in
// the same fixed order in every block (thread-strided sums, warp
// butterflies, warp 0 over the warp totals), so that all blocks of a launch
// obtain bitwise the same values; valid in thread 0.
template <int NQ>
__device__ __forceinline__ void all_blocks_sum_f32(const float* partials, int G, float (&out)[NQ]) {
    __shared__ float sh[NQ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = 0.0f;
    constexpr int BATCH = 8;  // loads issued together, then added in index order
    for (int k0 = threadIdx.x; k0 < G; k0 += BATCH * blockDim.x) {
        float x[NQ][BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int k = k0 + j * (int)blockDim.x;
#pragma unroll
            for (int q = 0; q < NQ; ++q) x[q][j] = k < G ? __ldg(partials + (size_t)q * G + k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j)
#pragma unroll
            for (int q = 0; q < NQ; ++q) t[q] += x[q][j];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        t[q] = warp_sum(t[q]);
        if (lane == 0) sh[q][warp] = t[q];
    }
    __syncthreads();
    if (warp == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = warp_sum(lane < nw ? sh[q][lane] : 0.0f);
    __syncthreads();  // sh is reused by the next call
}

// FP32 CG iteration in two or three launches (Chronopoulos-Gear form); the kernel
// boundaries serve as the grid-wide barriers. Step lengths (FP64):
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev).
// Two forms, chosen by the SpMV grid:
//  * deferred (a.defer, at most MIX_DEFER_MAX_BLOCKS blocks): k_mx_spmv leaves
//    per-block partials of the three dots; every block of k_mx_update (one
//    wave, rows strided) sums all of them in the same order, takes the stop
//    decision and forms the step lengths, so that no kernel has a last-block
//    reduction. The blocks of an update all read the previous step lengths,
//    so block 0 of the next k_mx_spmv commits the new ones;
//  * three launches (larger grids, where every block reading every partial would
//    cost more): k_mx_spmv leaves its partials, one block (k_mx_dots) sums them,
//    decides and commits, and k_mx_update_red4 reads the step lengths.

// FP32 SpMV row i: w = m u + dtau K32 u, and its terms of (r,u), (w,u), (r,r).
template <int F, int CH = 6>
__device__ __forceinline__ void mx_spmv_row(const MixArgs& a, int64_t i, float (&v)[3]) {
    const float u = a.Ul[i];
    const float w = fmaf((float)a.dtau, ell_row32<F, CH>(a.A, i, a.Ul), a.mass32[i] * u);
    const float res = a.Rl[i];
    a.Wl[i] = w;
    v[0] = res * u;
    v[1] = w * u;
    v[2] = res * res;
}

// FP32 update of row i: p = u + beta p; s = w + beta s; d += alpha p;
// r -= alpha s; u = D r (p = u, s = w in the first iteration).
__device__ __forceinline__ void mx_update_row(const MixArgs& a, int64_t i, float alpha, float beta, bool first) {
    const float u = a.Ul[i], w = a.Wl[i];
    const float p = first ? u : fmaf(beta, a.Pl[i], u);
    const float sp = first ? w : fmaf(beta, a.Sl[i], w);
    a.Pl[i] = p;
    a.Sl[i] = sp;
    a.Dl[i] = first ? alpha * p : fmaf(alpha, p, a.Dl[i]);
    const float res = fmaf(-alpha, sp, a.Rl[i]);
    a.Rl[i] = res;
    a.Ul[i] = res * a.Dinv[i];
}

// 8 blocks of 256 threads a SM (32 registers): the gathers of u are latency-bound, and at
// 5.75M rows a probe of this SpMV took 218 us at 8 blocks a SM against 244 us at 6.
// One block of the deferred-dot FP32 SpMV: block blk of a launch of nblk blocks for the
// machine of `a` (its own launch, or its range of a fused group launch).
template <int F, bool GROUP>
__device__ __forceinline__ void mx_spmv_block(const MixArgs& a, unsigned blk, unsigned nblk) {
    CgState* s = a.cg;
    if (s->done) {  // an iteration after the stop (rest of the loop body, host-driven lookahead)
        if (!GROUP && blk == 0) mx_done_on_entry(a);
        return;
    }
    if (blk == 0 && threadIdx.x == 0 && s->pending) {
        s->gamma = s->nx_gamma;
        s->alpha = s->nx_alpha;
        s->iter += 1;
        s->pending = 0;
    }
    float v[3] = {0.0f, 0.0f, 0.0f};
    const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    if (i < a.n) mx_spmv_row<F, GROUP ? 4 : 6>(a, i, v);
    block_partials_f32<3>(v, reinterpret_cast<float*>(a.partials), blk, nblk);
}

template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_mx_spmv(MixArgs a) {
    mx_spmv_block<F, false>(a, blockIdx.x, gridDim.x);
}

// One block of the FP32 CG update (deferred dots), block blk of nblk for the machine of
// `a`; in a fused group (GROUP) the stop clears the group's loop condition when the last
// member stops.
template <bool GROUP>
__device__ __forceinline__ void mx_update_block(const MixArgs& a, unsigned blk, unsigned nblk, const GroupArgs& g) {
    if (GROUP && a.ms->done) return;  // a member whose refinement converged in an earlier pass
    CgState* s = a.cg;
    __shared__ double prev[3];  // gamma_prev, alpha_prev, bb
    __shared__ float step[2];
    __shared__ int iter_sh, stop, skip;
    // Block 0 of this launch may set the stop flag while later blocks start:
    // one read per block, so that a block returns or proceeds as a whole.
    if (threadIdx.x == 0) {
        skip = s->done;
        iter_sh = s->iter;
        prev[0] = s->gamma;
        prev[1] = s->alpha;
        prev[2] = s->bb;
    }
    // the operands of the thread's first MX_UPDATE_ROWS rows are loaded before the dot
    // sums and the step lengths, so that their latency overlaps that chain; not by a
    // thread that already sees the stop flag (set by an earlier kernel, or by this
    // one's block 0 when it stops the solve, in which case no block updates rows)
    const int64_t stride = (int64_t)nblk * blockDim.x;
    const int64_t i0 = (int64_t)blk * blockDim.x + threadIdx.x;
    float u0[MX_UPDATE_ROWS], w0[MX_UPDATE_ROWS], p0[MX_UPDATE_ROWS], s0[MX_UPDATE_ROWS], d0[MX_UPDATE_ROWS],
        r0[MX_UPDATE_ROWS], q0[MX_UPDATE_ROWS];
    const bool live = !s->done;
#pragma unroll
    for (int k = 0; k < MX_UPDATE_ROWS; ++k) {
        const int64_t i = i0 + k * stride;
        u0[k] = w0[k] = p0[k] = s0[k] = d0[k] = r0[k] = q0[k] = 0.0f;
        if (i < a.n && live) {
            u0[k] = a.Ul[i];
            w0[k] = a.Wl[i];
            p0[k] = a.Pl[i];
            s0[k] = a.Sl[i];
            d0[k] = a.Dl[i];
            r0[k] = a.Rl[i];
            q0[k] = a.Dinv[i];
        }
    }
    __syncthreads();
    if (skip) {
        if (iter_sh == 0)  // the pass stopped before its first update: d = 0
            for (int64_t i = i0; i < a.n; i += stride) a.Dl[i] = 0.0f;
        return;
    }
    float out[3];
    all_blocks_sum_f32<3>(reinterpret_cast<const float*>(a.partials), a.part_blocks, out);
    const int iter = iter_sh;
    if (threadIdx.x == 0) {
        const double gamma = out[0], delta = out[1], rr = out[2];
        const bool st = rr <= prev[2] || iter >= a.max_iter;
        double alpha = 0.0, beta = 0.0;
        if (!st) {
            if (iter == 0) {
                alpha = gamma / delta;
            } else {
                beta = gamma / prev[0];
                alpha = gamma / (delta - beta * gamma / prev[1]);
            }
        }
        stop = st;
        step[0] = (float)alpha;
        step[1] = (float)beta;
        if (blk == 0) {
            s->runs += 1;
            *a.loop_kernels += 2;
            s->rr = rr;
            if (st) {
                *a.loop_kernels += 2 * (GROUP ? g.tail_pairs : a.tail_pairs);  // the rest of the body returns
                s->done = 1;
                if (GROUP) {
                    if (atomicSub(&g.gs->inner_active, 1) == 1)
                        cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_inner, 0u);
                } else if (a.h_inner) {
                    cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_inner, 0u);
                }
            } else {
                s->nx_gamma = gamma;
                s->nx_alpha = alpha;
                s->beta = beta;
                s->delta = delta;
                s->pending = 1;
                *a.iters_out += 1;
            }
        }
    }
    __syncthreads();
    if (stop) {
        if (iter == 0)  // the pass stopped before its first update: d = 0
            for (int64_t i = i0; i < a.n; i += stride) a.Dl[i] = 0.0f;
        return;
    }
    const float alpha = step[0], beta = step[1];
    const bool first = iter == 0;
#pragma unroll
    for (int k = 0; k < MX_UPDATE_ROWS; ++k) {
        const int64_t i = i0 + k * stride;
        if (i < a.n) {
            const float p = first ? u0[k] : fmaf(beta, p0[k], u0[k]);
            const float sp = first ? w0[k] : fmaf(beta, s0[k], w0[k]);
            a.Pl[i] = p;
            a.Sl[i] = sp;
            a.Dl[i] = first ? alpha * p : fmaf(alpha, p, d0[k]);
            const float res = fmaf(-alpha, sp, r0[k]);
            a.Rl[i] = res;
            a.Ul[i] = res * q0[k];
        }
    }
    for (int64_t i = i0 + MX_UPDATE_ROWS * stride; i < a.n; i += stride) mx_update_row(a, i, alpha, beta, first);
}

__global__ void __launch_bounds__(RED_BLOCK, 5) k_mx_update(MixArgs a) {
    mx_update_block<false>(a, blockIdx.x, gridDim.x, GroupArgs{});
}

// The decision of the large-grid FP32 CG from the grid's (r,u), (w,u), (r,r): stop test, or the
// step lengths that k_mx_update_red4 reads.
__device__ __forceinline__ void mx_red_commit(const MixArgs& a, const double (&out)[3]) {
    CgState* s = a.cg;
    s->runs += 1;
    *a.loop_kernels += a.pair_kernels;
    const double gamma = out[0], delta = out[1];
    s->rr = out[2];
    if (out[2] <= s->bb || s->iter >= a.max_iter) {
        *a.loop_kernels += a.pair_kernels * a.tail_pairs;  // the rest of the loop body runs and returns
        s->done = 1;
        if (a.h_inner) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_inner, 0u);
        return;
    }
    if (s->iter == 0) {
        s->beta = 0.0;
        s->alpha = gamma / delta;
    } else {
        const double beta = gamma / s->gamma;
        s->beta = beta;
        s->alpha = gamma / (delta - beta * gamma / s->alpha);
    }
    s->gamma = gamma;
    s->delta = delta;
    s->iter += 1;
    *a.iters_out += 1;
}

// The dots of the large-grid FP32 CG from k_mx_spmv's FP32 block partials: one block of
// MX_DOTS_THREADS sums every block's partial (thread t takes t, t + MX_DOTS_THREADS, ... in
// index order, in FP32 like the deferred form's sums; FP32 warp butterflies; FP64 over the warp
// sums) and commits. One SM's FP64 pipe is too narrow for 67k FP64 adds (54 us measured at
// 5.75M rows); in FP32 the kernel is a few round trips of loads. In a probe on the 5.75M-row
// FP32 structure (back-to-back SpMVs) the SpMV with stored partials took 175 us against 198 us
// with a last-block reduction in the SpMV itself, whose fence and atomic keep every block
// resident for a round trip more.
__global__ void __launch_bounds__(MX_DOTS_THREADS) k_mx_dots(MixArgs a) {
    if (a.cg->done) return;  // the SpMV counted the rest of the loop body
    const float* part = reinterpret_cast<const float*>(a.partials);
    const int G = a.part_blocks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float t[3] = {0.0f, 0.0f, 0.0f};
    constexpr int BATCH = 8;  // loads issued together, then added in index order
    for (int k0 = threadIdx.x; k0 < G; k0 += BATCH * MX_DOTS_THREADS) {
        float x[3][BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int k = k0 + j * MX_DOTS_THREADS;
#pragma unroll
            for (int q = 0; q < 3; ++q) x[q][j] = k < G ? __ldg(part + (size_t)q * G + k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) t[q] += x[q][j];
    }
    __shared__ double sh[3][32];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        t[q] = warp_sum(t[q]);
        if (lane == 0) sh[q][warp] = (double)t[q];
    }
    __syncthreads();
    if (warp == 0) {
        double out[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) out[q] = warp_sum(sh[q][lane]);
        if (lane == 0) mx_red_commit(a, out);
    }
}

__global__ void k_mx_update_red(MixArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.cg->done) {
        if (a.cg->iter == 0 && i < a.n) a.Dl[i] = 0.0f;  // the pass stopped before its first update
        return;
    }
    if (i < a.n) mx_update_row(a, i, (float)a.cg->alpha, (float)a.cg->beta, a.cg->iter == 1);
}

// k_mx_update_red on four consecutive rows a thread with 16-byte loads and stores (vectors
// 16-byte aligned): four times the bytes in flight a thread, the arithmetic of mx_update_row
// on every row. The last rows, past the last multiple of four, take mx_update_row.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& c4(float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__global__ void k_mx_update_red4(MixArgs a) {
    const int64_t i0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= a.n) return;
    if (a.cg->done) {
        if (a.cg->iter == 0)
            for (int64_t i = i0; i < min(i0 + 4, a.n); ++i) a.Dl[i] = 0.0f;
        return;
    }
    const float alpha = (float)a.cg->alpha, beta = (float)a.cg->beta;
    const bool first = a.cg->iter == 1;
    if (i0 + 4 > a.n) {
        for (int64_t i = i0; i < a.n; ++i) mx_update_row(a, i, alpha, beta, first);
        return;
    }
    const float4 u = ld4(a.Ul + i0), w = ld4(a.Wl + i0), rr = ld4(a.Rl + i0), di = ld4(a.Dinv + i0);
    float4 p = u, sp = w, d = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!first) {
        p = ld4(a.Pl + i0);
        sp = ld4(a.Sl + i0);
        d = ld4(a.Dl + i0);
    }
    float4 res, un;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 uu = u, ww = w, r4 = rr, dd = di;
        const float pk = first ? c4(uu, k) : fmaf(beta, c4(p, k), c4(uu, k));
        const float sk = first ? c4(ww, k) : fmaf(beta, c4(sp, k), c4(ww, k));
        c4(p, k) = pk;
        c4(sp, k) = sk;
        c4(d, k) = first ? alpha * pk : fmaf(alpha, pk, c4(d, k));
        const float rk = fmaf(-alpha, sk, c4(r4, k));
        c4(res, k) = rk;
        c4(un, k) = rk * c4(dd, k);
    }
    st4(a.Pl + i0, p);
    st4(a.Sl + i0, sp);
    st4(a.Dl + i0, d);
    st4(a.Rl + i0, res);
    st4(a.Ul + i0, un);
}

// End of a refinement pass: x += d and r -= A d, with r and x in FP64. The
// residual r = b - A x of the corrected iterate is thereby carried as
//   r = r0 - A (x - x0),
// r0 = b - A x0 formed in FP64 (k_mx_init); only the correction-sized term
// A d of a pass is applied with the FP32 operator (an FP32 SpMV of d), so its
// rounding is relative to the correction, not to b. Outer stop test.
// One block of the end of a refinement pass (see k_mx_refine), block blk of nblk for the
// machine of `a`; in a fused group the outer loop stops with the last member's convergence.
template <int F, bool GROUP>
__device__ __forceinline__ void mx_refine_block(const MixArgs& a, unsigned blk, unsigned nblk, const GroupArgs& g) {
    if (GROUP && a.ms->done) return;  // a member whose refinement converged in an earlier pass
    double v[1] = {0.0};
    const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const float d = a.Dl[i];
        a.X[i] += (double)d;
        a.Dsum[i] += d;
        const float Ad = fmaf((float)a.dtau, ell_row32<F, GROUP ? 4 : 6>(a.A, i, a.Dl), a.mass32[i] * d);
        const double res = a.R[i] - (double)Ad;
        a.R[i] = res;
        a.Rl[i] = (float)res;  // the next pass's FP32 residual and u (unread if none follows)
        a.Ul[i] = (float)res * a.Dinv[i];
        v[0] += res * res;
    }
    double out[1];
    if (reduce_last2_at<1>(v, a.partials, a.gpartials, a.counter, out, blk, nblk) && threadIdx.x == 0) {
        MixState* s = a.ms;
        s->rr = out[0];
        s->passes += 1;
        *a.loop_kernels += 1;
        *a.refine_out = s->passes;
        const bool conv = out[0] <= a.rtol2 * s->bb;
        if (conv || s->passes >= a.max_refine) {
            s->done = 1;
            if (!conv) report_status(a.status, SDC_ERR_NOT_CONVERGED);
            if (GROUP) {
                if (atomicSub(&g.gs->outer_active, 1) == 1)
                    cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_outer, 0u);
            } else if (a.h_outer) {
                cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer, 0u);
            }
        } else {
            mx_begin_pass(a, out[0]);
            if (GROUP) cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_inner, 1u);
        }
    }
}

template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_mx_refine(MixArgs a) {
    mx_refine_block<F, false>(a, blockIdx.x, gridDim.x, GroupArgs{});
}

// Fused group launches: the member of each block and its block within the member's range.
__device__ __forceinline__ const MixArgs& group_member(const GroupArgs& g, const GroupLaunch& L, unsigned& blk,
                                                       unsigned& nblk) {
    const int m = L.member[blockIdx.x];
    const int f = L.first[m];
    blk = blockIdx.x - (unsigned)f;
    nblk = (unsigned)(L.first[m + 1] - f);
    return g.args[m];
}

// Start of a fused group's solve, after every member's k_mx_init: the refinement loop runs
// if any member has a pass to do.
__global__ void k_group_begin(GroupArgs g) {
    if (threadIdx.x == 0) {
        g.gs->passes = 0;
        g.gs->launches = 0;
        cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_outer, g.gs->outer_active > 0 ? 1u : 0u);
    }
}

// End of a fused group's solve: the counters start the next solve at zero, whatever ended
// this one.
__global__ void k_group_end(GroupArgs g) {
    if (threadIdx.x == 0) {
        g.gs->outer_active = 0;
        g.gs->inner_active = 0;
    }
}

// The group's loops must end even if no member stops them: a caps count failure of the
// group (every member's status gets SDC_ERR_NOT_CONVERGED).
__device__ __forceinline__ void group_cap_failed(const GroupArgs& g) {
    for (int m = 0; m < g.n_members; ++m) report_status(g.args[m].status, SDC_ERR_NOT_CONVERGED);
}

template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_mx_spmv_g(GroupArgs g) {
    // the inner loop ends after this body when no member's CG runs (the counter changes only
    // in the updates, outside this launch) or after launch_cap SpMV launches in the pass
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int n = ++g.gs->launches;
        if (g.gs->inner_active <= 0 || n > g.launch_cap) {
            cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_inner, 0u);
            if (n > g.launch_cap) group_cap_failed(g);
        }
    }
    unsigned blk, nblk;
    const MixArgs& a = group_member(g, g.spmv, blk, nblk);
    mx_spmv_block<F, true>(a, blk, nblk);
}

__global__ void __launch_bounds__(RED_BLOCK, 5) k_mx_update_g(GroupArgs g) {
    unsigned blk, nblk;
    const MixArgs& a = group_member(g, g.update, blk, nblk);
    mx_update_block<true>(a, blk, nblk, g);
}

template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_mx_refine_g(GroupArgs g) {
    // the outer loop ends after this pass when no member is refining or after pass_cap passes
    // (members that go on set the inner loop's condition again for their next pass)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int n = ++g.gs->passes;
        g.gs->launches = 0;
        if (g.gs->outer_active <= 0 || n >= g.pass_cap) {
            cudaGraphSetConditional((cudaGraphConditionalHandle)g.h_outer, 0u);
            if (n >= g.pass_cap && g.gs->outer_active > 0) group_cap_failed(g);
        }
    }
    unsigned blk, nblk;
    const MixArgs& a = group_member(g, g.refine, blk, nblk);
    mx_refine_block<F, true>(a, blk, nblk, g);
}

// Diagnostics of a mixed solve: the true residual ||b - (m x + dtau K x)|| / ||b|| with the
// FP64 operator and the FP64 iterate, after the refinement stopped on the carried residual.
template <bool C32>
__global__ void k_mx_true_residual(MixArgs a) {
    double v[2] = {0.0, 0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const double b = a.B[i];
        const double r = b - fma(a.dtau, ell_row<C32>(a.A, i, a.X), a.mass[i] * a.X[i]);
        v[0] = r * r;
        v[1] = b * b;
    }
    double out[2];
    if (reduce_last2<2>(v, a.partials, a.gpartials, a.counter, out) && threadIdx.x == 0)
        *a.true_res = out[1] > 0.0 ? sqrt(out[0] / out[1]) : sqrt(out[0]);
}

// ------------------------------------------------------------------ endpoint

// f*_m = f^I(T*) + g (Algorithm 1) or f^I(T*) - f^I(T^k_m) (Algorithm 2), and
// the endpoint T_{m,P} of every DOF off the contact, where f^E vanishes and
// the P explicit substeps add up exactly to
//   m T_{m,P} = m T_{m-1} + dtau f*_m + sum_j dt s_{m,j} F^I_j
// (sum_p stil_{m,p,j} = s_{m,j}). Contact rows are overwritten by the
// substep loop that follows.
// The row a thread of a bulk-endpoint launch handles (BulkArgs::rows), or -1.
__device__ __forceinline__ int64_t bulk_row(const BulkArgs& a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.rows == BULK_CONTACT) return t < a.n_iface ? (int64_t)a.dof[t] : -1;
    if (t >= a.n) return -1;
    return (a.rows == BULK_OFF_CONTACT && a.pos[t] >= 0) ? -1 : t;
}

template <bool C32>
__global__ void k_bulk_endpoint(BulkArgs a) {
    const int64_t i = bulk_row(a);
    if (i >= 0) {
        const double KX = ell_row<C32>(a.A, i, a.X);
        double incr, fstar;
        if (a.mode == RHS_PRED) {
            fstar = a.g[i] - KX;
            incr = a.dtau * fstar;
        } else {
            fstar = -KX - (a.FIm[i] - a.g[i]);
            double I = 0.0;
            for (int j = 0; j < a.nFI; ++j) I = fma(a.Sdt[j], a.FI[j][i], I);
            incr = fma(a.dtau, fstar, I);
        }
        const int pa = a.pos[i];
        if (pa >= 0) a.fstar_I[pa] = fstar;  // contact rows: T_m comes from the substep loop
        else a.Tout[i] = fma(incr, a.minv[i], a.Tprev[i]);
    }
}

// Mixed precision form of k_bulk_endpoint (see BulkArgs): with T* = x0 + dX,
//   predictor: f*_m = F^I(T*) + g = F(x0) - K dX
//   sweep:     f*_m = f^I(T*) - f^I(T^k_m) = -K dX          (x0 = T^k_m)
// K dX as an FP32 SpMV; the increment of every row goes to dT for k_fi_mx.
template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_bulk_endpoint_mx(BulkArgs a) {
    const int64_t i = bulk_row(a);
    if (i >= 0) {
        const double KdX = (double)ell_row32<F>(a.A, i, a.dX);
        double incr, fstar;
        if (a.mode == RHS_PRED) {
            fstar = a.Fx0[i] - KdX;
            incr = a.dtau * fstar;
        } else {
            fstar = -KdX;
            double I = 0.0;
            for (int j = 0; j < a.nFI; ++j) I = fma(a.Sdt[j], a.FI[j][i], I);
            incr = fma(a.dtau, fstar, I);
        }
        const int pa = a.pos[i];
        if (pa >= 0) {
            a.fstar_I[pa] = fstar;  // contact rows: T_m and its increment come from the substep loop
        } else {
            const double dT = incr * a.minv[i];
            a.Tout[i] = a.Tprev[i] + dT;
            a.dT[i] = (float)dT;
        }
    }
}

// F^I(T_m) + g = F^I(T_prev) + g - K dT (mixed precision; FP32 SpMV of the increment)
template <int F>
__global__ void __launch_bounds__(RED_BLOCK, 8) k_fi_mx(FiDevArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) a.F[i] = a.Fprev[i] - (double)ell_row32<F>(a.A, i, a.dT);
}

// Both column forms of every kernel that reads the matrix (EllDev), for the host code of
// other translation units (the stubs of template kernels are local to this one)
#define SDC_MATRIX_KERNEL(name, type) \
    type name##_form(bool c32) { return c32 ? name<true> : name<false>; }
SDC_MATRIX_KERNEL(k_apply_operator, KEllOp)
SDC_MATRIX_KERNEL(k_fi, KEllFi)
SDC_MATRIX_KERNEL(k_cg_init, KCgInit)
SDC_MATRIX_KERNEL(k_ie_init, KCgInit)
SDC_MATRIX_KERNEL(k_cg_spmv, KCg)
SDC_MATRIX_KERNEL(k_ie_spmv, KCg)
SDC_MATRIX_KERNEL(k_mx_init, KMxInit)
SDC_MATRIX_KERNEL(k_mx_true_residual, KMx)
SDC_MATRIX_KERNEL(k_bulk_endpoint, KBulk)
#undef SDC_MATRIX_KERNEL
// The kernels that read only the FP32 copy, in its three forms (0 = 16-bit offsets,
// 1 = 32-bit columns, 2 = implied columns)
#define SDC_MATRIX32_KERNEL(name, type) \
    type name##_form32(int f) { return f == 2 ? name<2> : f == 1 ? name<1> : name<0>; }
SDC_MATRIX32_KERNEL(k_mx_spmv, KMx)
SDC_MATRIX32_KERNEL(k_mx_refine, KMx)
SDC_MATRIX32_KERNEL(k_mx_spmv_g, KGroup)
SDC_MATRIX32_KERNEL(k_mx_refine_g, KGroup)
SDC_MATRIX32_KERNEL(k_bulk_endpoint_mx, KBulk)
SDC_MATRIX32_KERNEL(k_fi_mx, KFi)
#undef SDC_MATRIX32_KERNEL

// ------------------------------------------------------------------ contact geometry

__device__ __forceinline__ void motion_at(const ContactDev& C, double tau, double& du, double& dv, double& q) {
    const double ph = 2.0 * 3.14159265358979323846 * tau / C.period;
    const double s = __dadd_rn(C.z0, __dmul_rn(C.amp, sin(ph)));
    du = C.dir_u * s;
    dv = C.dir_v * s;
    q = C.q0 * fabs(cos(ph));
}

// Merge c into the row's entry for `node` (entry k of this thread at idx[k * GEOM_THREADS]).
template <typename R>
__device__ __forceinline__ void add_entry(int32_t* idx, R* coef, int& n, int node, R c, bool& overflow) {
    for (int k = 0; k < n; ++k)
        if (idx[k * GEOM_THREADS] == node) {
            coef[k * GEOM_THREADS] += c;
            return;
        }
    if (n < MAXE) {
        idx[n * GEOM_THREADS] = node;
        coef[n * GEOM_THREADS] = c;
        ++n;
    } else {
        overflow = true;
    }
}

// Coupling operator of Sec. 2 at one substep time, row by row:
//   f^E_a = sum over faces Q containing a, faces R of the other body
//           overlapping Q, of the 2x2 Gauss rule on the overlap of
//           phi^Q_a (h_c (T_R - T_Q) + q/2),
// stored as a constant plus coefficients on contact DOFs. Shape functions
// of axis-aligned bilinear faces are products of linear functions of u and
// of v, and the 2x2 rule is the product of two 2-point rules, so every
// coefficient is a product of two one-dimensional sums:
//   int phi^Q_a phi^X_c = [sum_g w_g l^Q_a(u_g) l^X_c(u_g)] [sum_g w_g l^Q_a(v_g) l^X_c(v_g)].
// The search for overlapping faces and the overlap bounds are FP64. The
// integrals take coordinates relative to the low corner of Q (formed in
// FP64) and run in R: FP64 for the FP64 path; FP32 for mixed precision,
// whose coefficients enter only through products with temperature
// differences (see k_iface_prep), on GB300's wide FP32 pipes instead of
// its narrow FP64 pipe.
template <typename R>
__device__ __forceinline__ void iface_geom_impl(const GeomArgs& g) {
    const ContactDev& C = g.C;
    const int NI = C.n_iface;
    const int s = (int)blockIdx.y;
    const int a = (int)(blockIdx.x * GEOM_THREADS + threadIdx.x);
    // the slot's motion, once per block
    __shared__ double mot[3];
    __shared__ int32_t s_idx[MAXE * GEOM_THREADS];
    __shared__ R s_coef[MAXE * GEOM_THREADS];
    if (threadIdx.x == 0) {
        double tau;
        if (g.use_fixed) {
            tau = g.t_fixed;
        } else {
            const double tn = __dadd_rn(g.st->t0, __dmul_rn((double)g.st->n_done, g.st->dt));
            tau = __dadd_rn(tn, __dmul_rn(g.st->dt, g.slot_pos[s]));
        }
        motion_at(C, tau, mot[0], mot[1], mot[2]);
    }
    __syncthreads();
    if (a >= NI) return;
    const double du = mot[0], dv = mot[1];
    const R q = (R)mot[2];
    int32_t* idx = s_idx + threadIdx.x;
    R* coef = s_coef + threadIdx.x;
    const bool stock = a >= C.n_iface_fix;
    const R h_c = (R)C.h_c;
    {
        // no face of this DOF can touch the other body's contact faces: empty row
        Rect4 mine = C.dof_box[a], other = stock ? C.box_fix : C.box_mov;
        if (stock) {
            mine.x += du; mine.z += du; mine.y += dv; mine.w += dv;
        } else {
            other.x += du; other.z += du; other.y += dv; other.w += dv;
        }
        if (!(fmin(mine.z, other.z) > fmax(mine.x, other.x) && fmin(mine.w, other.w) > fmax(mine.y, other.y))) {
            const size_t so = (size_t)s * NI + a;
            g.E.cnt[so] = 0;
            g.E.cst[so] = 0.0;
            return;
        }
    }
    const R gp = (R)0.57735026918962576451;  // 1/sqrt(3)

    int n = 0;
    bool overflow = false;
    R cst = 0;
    const BinsDev& B = stock ? C.bins_fix : C.bins_mov;
    for (int e = C.inc_ptr[a]; e < C.inc_ptr[a + 1]; ++e) {
        const int Qf = C.inc_quad[e];
        const int code = C.inc_code[e];
        const int au = code & 1, av = code >> 1;
        Rect4 Q = C.rect[Qf];
        if (stock) {
            Q.x += du; Q.z += du; Q.y += dv; Q.w += dv;
        }
        const double2 qi = C.rinv[Qf];
        const R qix = (R)qi.x, qiy = (R)qi.y;
        const R qwu = (R)(Q.z - Q.x), qwv = (R)(Q.w - Q.y);
        const int4 qn = C.qnode[Qf];
        // query rectangle in the partner body's frame (stock partners are in reference position)
        const double su = stock ? 0.0 : du, sv = stock ? 0.0 : dv;
        const double lo_u = Q.x - su, lo_v = Q.y - sv, hi_u = Q.z - su, hi_v = Q.w - sv;
        // a partner's low corner lies in (lo - bin, hi) along each axis (bins are at least one face
        // wide); the 1e-9 bin margin absorbs the rounding of these quotients
        int iu0 = (int)floor((lo_u - B.bu - B.ou) * B.ibu - 1e-9), iu1 = (int)floor((hi_u - B.ou) * B.ibu + 1e-9);
        int iv0 = (int)floor((lo_v - B.bv - B.ov) * B.ibv - 1e-9), iv1 = (int)floor((hi_v - B.ov) * B.ibv + 1e-9);
        iu0 = max(iu0, 0); iv0 = max(iv0, 0);
        iu1 = min(iu1, B.nu - 1); iv1 = min(iv1, B.nv - 1);
        for (int iv = iv0; iv <= iv1; ++iv)
            for (int iu = iu0; iu <= iu1; ++iu) {
                const int bin = iv * B.nu + iu;
                for (int t = B.ptr[bin]; t < B.ptr[bin + 1]; ++t) {
                    const int Rf = B.item[t];
                    Rect4 Rr = C.rect[Rf];
                    R ua_, ub_, va_, vb_, rlu, rhu, rlv, rhv;
                    if constexpr (std::is_same<R, float>::value) {
                        // mixed: four FP64 differences to the low corner of Q in the partner's
                        // frame (qlu = Q.x - shift), then FP32; the overlap test keeps its sign
                        // exactly (a rounded difference is zero only when the FP64 one is)
                        const double qlu = Q.x - su, qlv = Q.y - sv;
                        rlu = (R)(Rr.x - qlu);
                        rhu = (R)(Rr.z - qlu);
                        rlv = (R)(Rr.y - qlv);
                        rhv = (R)(Rr.w - qlv);
                        ua_ = fmaxf(R(0), rlu);
                        ub_ = fminf(qwu, rhu);
                        va_ = fmaxf(R(0), rlv);
                        vb_ = fminf(qwv, rhv);
                        if (!(ub_ > ua_ && vb_ > va_)) continue;
                    } else {
                        if (!stock) {
                            Rr.x += du; Rr.z += du; Rr.y += dv; Rr.w += dv;
                        }
                        const double ua = fmax(Q.x, Rr.x), ub = fmin(Q.z, Rr.z);
                        const double va = fmax(Q.y, Rr.y), vb = fmin(Q.w, Rr.w);
                        if (!(ub > ua && vb > va)) continue;
                        // coordinates relative to the low corner of Q
                        ua_ = (R)(ua - Q.x); ub_ = (R)(ub - Q.x); va_ = (R)(va - Q.y); vb_ = (R)(vb - Q.y);
                        rlu = (R)(Rr.x - Q.x); rhu = (R)(Rr.z - Q.x); rlv = (R)(Rr.y - Q.y); rhv = (R)(Rr.w - Q.y);
                    }
                    const double2 ri = C.rinv[Rf];
                    const R rix = (R)ri.x, riy = (R)ri.y;
                    const int4 rn = C.qnode[Rf];
                    const R hu = R(0.5) * (ub_ - ua_), hv = R(0.5) * (vb_ - va_);
                    const R cu = R(0.5) * (ua_ + ub_), cv = R(0.5) * (va_ + vb_);
                    const R u[2] = {cu - gp * hu, cu + gp * hu};
                    const R v[2] = {cv - gp * hv, cv + gp * hv};
                    // linear factors at the Gauss abscissae: index 0 = low-side node, 1 = high-side node
                    R lqu[2][2], lru[2][2], lqv[2][2], lrv[2][2];
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        lqu[1][k] = u[k] * qix;
                        lqu[0][k] = (qwu - u[k]) * qix;
                        lru[1][k] = (u[k] - rlu) * rix;
                        lru[0][k] = (rhu - u[k]) * rix;
                        lqv[1][k] = v[k] * qiy;
                        lqv[0][k] = (qwv - v[k]) * qiy;
                        lrv[1][k] = (v[k] - rlv) * riy;
                        lrv[0][k] = (rhv - v[k]) * riy;
                    }
                    R iqu[2], iru[2], iqv[2], irv[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        iqu[c] = hu * fma(lqu[au][0], lqu[c][0], lqu[au][1] * lqu[c][1]);
                        iru[c] = hu * fma(lqu[au][0], lru[c][0], lqu[au][1] * lru[c][1]);
                        iqv[c] = hv * fma(lqv[av][0], lqv[c][0], lqv[av][1] * lqv[c][1]);
                        irv[c] = hv * fma(lqv[av][0], lrv[c][0], lqv[av][1] * lrv[c][1]);
                    }
                    cst += R(0.5) * q * (hu * (lqu[au][0] + lqu[au][1])) * (hv * (lqv[av][0] + lqv[av][1]));
                    const int qnc[4] = {qn.x, qn.y, qn.z, qn.w};
                    const int rnc[4] = {rn.x, rn.y, rn.z, rn.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        add_entry<R>(idx, coef, n, qnc[c], -h_c * iqu[c & 1] * iqv[c >> 1], overflow);
                        add_entry<R>(idx, coef, n, rnc[c], h_c * iru[c & 1] * irv[c >> 1], overflow);
                    }
                }
            }
    }
    if (overflow) report_status(g.status, SDC_ERR_ARG);
    const size_t so = (size_t)s * NI + a;
    g.E.cnt[so] = n;
    g.E.cst[so] = (double)cst;
    for (int k = 0; k < n; ++k) {
        const size_t o = ((size_t)s * MAXE + k) * NI + a;
        const int j = idx[k * GEOM_THREADS];
        g.E.idx[o] = j;
        const R cf = coef[k * GEOM_THREADS];
        if (g.E.coef) g.E.coef[o] = (double)cf;
        if (g.E.coef32) g.E.coef32[o] = (float)cf;
    }
}

__global__ void __launch_bounds__(GEOM_THREADS) k_iface_geom(GeomArgs g) { iface_geom_impl<double>(g); }

__global__ void __launch_bounds__(GEOM_THREADS) k_iface_geom_mx(GeomArgs g) { iface_geom_impl<float>(g); }

__device__ __forceinline__ double apply_coupling(const CouplingOp& E, int slot, int NI, int a, const double* T) {
    const size_t so = (size_t)slot * NI + a;
    const int n = E.cnt[so];
    double acc = E.cst[so];
    for (int k = 0; k < n; ++k) {
        const size_t o = ((size_t)slot * MAXE + k) * NI + a;
        acc = fma(__ldg(E.coef + o), __ldcg(T + __ldg(E.idx + o)), acc);
    }
    return acc;
}

// Coupling entries of one contact DOF at one slot, the first B loaded ahead
// of use (the operator does not depend on T, so these loads can be issued
// before the wait that publishes T).
template <int B>
struct CouplingRowT {
    int n;
    double cst;
    int idx[B];
    double coef[B];
};
using CouplingRow = CouplingRowT<IFACE_BATCH>;

template <int B>
__device__ __forceinline__ void coupling_prefetch(const CouplingOp& E, int slot, int NI, int a, CouplingRowT<B>& r) {
    const size_t so = (size_t)slot * NI + a;
    r.n = __ldg(E.cnt + so);
    r.cst = __ldg(E.cst + so);
#pragma unroll
    for (int k = 0; k < B; ++k) {  // entries past n are never used
        const size_t o = ((size_t)slot * MAXE + k) * NI + a;
        r.idx[k] = __ldg(E.idx + o);
        r.coef[k] = __ldg(E.coef + o);
    }
}

// cst + sum_k coef_k T[idx_k] on a replica of T_I in this CTA's shared memory,
// in entry order; the entries past the prefetched batch are fetched 16 at a
// time with all loads of a round issued together.
// replica element: shared memory, or global memory written by other CTAs (read through L2)
template <bool GL, typename V>
__device__ __forceinline__ V rep_load(const V* p) {
    if constexpr (GL) return __ldcg(p);
    else return *p;
}

template <int B, bool GL = false>
__device__ __forceinline__ double coupling_apply_shared(const CouplingOp& E, int slot, int NI, int a,
                                                        const CouplingRowT<B>& r, const double* Tsh) {
    constexpr int B2 = 16;  // later rounds
    double acc = r.cst;
#pragma unroll
    for (int k = 0; k < B; ++k)
        if (k < r.n) acc = fma(r.coef[k], rep_load<GL>(Tsh + r.idx[k]), acc);
    for (int k0 = B; k0 < r.n; k0 += B2) {
        int id[B2];
        double cf[B2];
#pragma unroll
        for (int j = 0; j < B2; ++j) {
            const int k = k0 + j;
            if (k < r.n) {
                const size_t o = ((size_t)slot * MAXE + k) * NI + a;
                id[j] = __ldg(E.idx + o);
                cf[j] = __ldg(E.coef + o);
            }
        }
#pragma unroll
        for (int j = 0; j < B2; ++j)
            if (k0 + j < r.n) acc = fma(cf[j], rep_load<GL>(Tsh + id[j]), acc);
    }
    return acc;
}

// FP32 coupling entries of one contact DOF at one slot (mixed precision).
template <int B>
struct CouplingRow32T {
    int n;
    int idx[B];
    float coef[B];
};

template <int B>
__device__ __forceinline__ void coupling_prefetch32(const CouplingOp& E, int slot, int NI, int a, CouplingRow32T<B>& r) {
    r.n = __ldg(E.cnt + (size_t)slot * NI + a);
#pragma unroll
    for (int k = 0; k < B; ++k) {  // entries past n are never used
        const size_t o = ((size_t)slot * MAXE + k) * NI + a;
        r.idx[k] = __ldg(E.idx + o);
        r.coef[k] = __ldg(E.coef32 + o);
    }
}

// sum_k coef32_k dT[idx_k] in FP32 on a shared-memory replica of the deviations dT
template <int B, bool GL = false>
__device__ __forceinline__ float coupling_apply_shared32(const CouplingOp& E, int slot, int NI, int a,
                                                         const CouplingRow32T<B>& r, const float* dT) {
    constexpr int B2 = 16;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < B; ++k)
        if (k < r.n) acc = fmaf(r.coef[k], rep_load<GL>(dT + r.idx[k]), acc);
    for (int k0 = B; k0 < r.n; k0 += B2) {
        int id[B2];
        float cf[B2];
#pragma unroll
        for (int j = 0; j < B2; ++j) {
            const int k = k0 + j;
            if (k < r.n) {
                const size_t o = ((size_t)slot * MAXE + k) * NI + a;
                id[j] = __ldg(E.idx + o);
                cf[j] = __ldg(E.coef32 + o);
            }
        }
#pragma unroll
        for (int j = 0; j < B2; ++j)
            if (k0 + j < r.n) acc = fmaf(cf[j], rep_load<GL>(dT + id[j]), acc);
    }
    return acc;
}

// f^E(T, tau) on all DOFs for one precomputed slot (zero elsewhere is set by the caller).
__global__ void k_contact_apply(ContactDev C, CouplingOp E, int slot, const double* __restrict__ T,
                                double* __restrict__ Ti, double* __restrict__ out, int phase) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= C.n_iface) return;
    if (phase == 0) {
        Ti[a] = T[C.dof[a]];
    } else {
        out[C.dof[a]] = apply_coupling(E, slot, C.n_iface, a, Ti);
    }
}

// ------------------------------------------------------------------ single-rate SDC

// f^E(T, tau) on the contact DOFs at one slot of the step's coupling operator
// (single-rate SDC evaluates f^E only at the standard nodes, which are the end
// slots of the intervals). One thread per contact DOF; coupling indices are
// contact DOFs.
__global__ void k_sisdc_fe(SisdcArgs a) {
    const int NI = a.C.n_iface;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NI) return;
    const size_t so = (size_t)a.slot * NI + i;
    const int n = a.E.cnt[so];
    const double Ta = a.T[a.C.dof[i]];
    double acc = a.E.cst[so];
    for (int k = 0; k < n; ++k) {
        const size_t o = ((size_t)a.slot * MAXE + k) * NI + i;
        const double Tj = a.T[a.C.dof[a.E.idx[o]]];
        // mixed precision: zero-sum FP32 rows applied to differences (see k_iface_prep)
        acc = a.E.coef32 ? fma((double)a.E.coef32[o], Tj - Ta, acc) : fma(a.E.coef[o], Tj, acc);
    }
    a.fe_out[i] = acc;
}

// The contact-row terms of the implicit stage of single-rate SDC (Sec. 3):
//   predictor: dtau f^E(T_{m-1}, tau_{m-1})
//   sweep:     dtau (f^E(T^{k+1}_{m-1}) - f^E(T^k_{m-1})) + sum_j dt s_{m,j} f^E(T^k_j, tau_j)
// (the f^I + g part of the quadrature is added by the solve's RHS).
__global__ void k_sisdc_rhs(SisdcArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.C.n_iface) return;
    double v;
    if (a.mode == RHS_PRED) {
        v = a.dtau * a.fe_left_new[i];
    } else {
        v = a.dtau * (a.fe_left_new[i] - a.fe_left_old[i]);
        for (int j = 0; j < a.nFE; ++j) v = fma(a.Sdt[j], a.fe_old[j][i], v);
    }
    a.ihat[i] = v;
}

// T_m = the implicit stage's solution on every row; its increment in FP32 for
// the mixed-precision F^I update (may be NULL).
__global__ void k_sisdc_endpoint(const double* __restrict__ X, const double* __restrict__ Tprev,
                                 double* __restrict__ Tout, float* __restrict__ dT, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = X[i];
    Tout[i] = x;
    if (dT) dT[i] = (float)(x - Tprev[i]);
}

// ------------------------------------------------------------------ substep loop

__device__ __forceinline__ double substep_dt(const IfaceArgs& a, double tn, int p) {
    return __dadd_rn(tn, __dmul_rn(a.dt, a.emb[p])) - __dadd_rn(tn, __dmul_rn(a.dt, a.emb[p - 1]));
}

// T on the contact DOFs by contact index, Tc[i] = T[dof[i]]: the gathers of k_iface_prep then
// take one load a coupling entry instead of two dependent ones.
__global__ void k_iface_tc(ContactDev C, const double* __restrict__ T, double* __restrict__ Tc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.n_iface) Tc[i] = T[C.dof[i]];
}

// c_p of every substep and contact DOF (see PrepArgs); one thread per (p, DOF),
// p = 0..P (p = 0 only forms base_0 in mixed precision).
// Length of substep p of the interval of a k_iface_prep launch (the embedded nodes' times at
// this step, as the substep loop forms them).
__device__ __forceinline__ double prep_dtp(const PrepArgs& a, int p) {
    const double tn = __dadd_rn(a.st->t0, __dmul_rn((double)a.st->n_done, a.st->dt));
    return __dadd_rn(tn, __dmul_rn(a.dt, a.emb[p])) - __dadd_rn(tn, __dmul_rn(a.dt, a.emb[p - 1]));
}

__global__ void k_iface_prep(PrepArgs a) {
    const int NI = a.C.n_iface;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the substep lengths of this block's rows: with NI >= blockDim a block spans at most two
    // substeps, whose lengths (a dozen FP64 operations, on GB300's narrow FP64 pipe) are formed
    // once per block; smaller interfaces form them per thread
    const bool per_block = NI >= (int)blockDim.x;
    __shared__ double s_dtp[2];
    const int p_first = (int)(((int64_t)blockIdx.x * blockDim.x) / NI);
    if (per_block && threadIdx.x < 2) {
        const int pp = p_first + (int)threadIdx.x;
        if (pp >= 1 && pp <= a.P) s_dtp[threadIdx.x] = prep_dtp(a, pp);
    }
    __syncthreads();
    if (gid >= (int64_t)NI * (a.P + 1)) return;
    const int p = (int)(gid / NI), i = (int)(gid % NI);
    if (a.base) {
        // f^E(T_{m-1}, tau_{m,p}) in FP64 from the FP32 coefficients: the exchange
        // coefficients of a row sum to zero (both bodies' shape functions are partitions of
        // unity on every overlap), so f^E = cst + sum_k coef_k (T_k - T_a) exactly, and the
        // coefficients' rounding multiplies temperature differences, not the temperature
        const int slot = a.slot0 + p;
        const size_t so = (size_t)slot * NI + i;
        const int n = a.E.cnt[so];
        const double Ta = a.Tc[i];
        double acc = a.E.cst[so];
        for (int k = 0; k < n; ++k) {
            const size_t o = ((size_t)slot * MAXE + k) * NI + i;
            const int j = a.E.idx[o];
            acc = fma((double)a.E.coef32[o], a.Tc[j] - Ta, acc);
        }
        a.base[(size_t)p * NI + i] = acc;
    }
    if (p == 0 || a.mode == RHS_PRED) return;  // Algorithm 1: c_p = dt_p f*_m (formed by the loop)
    const double dtp = per_block ? s_dtp[p - p_first] : prep_dtp(a, p);
    const int row = a.C.dof[i];
    double I = 0.0;
    for (int j = 0; j < a.nFI; ++j) I = fma(a.Stil[(size_t)(p - 1) * a.nFI + j], a.FI[j][row], I);
    // the embedded quadrature's row is windowed (M nonzero weights of P): zero weights are
    // skipped by an integer test of their bits (a -0.0 weight adds -0.0 to a sum that starts at
    // +0.0 and changes nothing), not by an FP64 compare
    for (int qq = 1; qq <= a.P; ++qq) {
        const double wq = a.Semb[(size_t)(p - 1) * a.P + (qq - 1)];
        if (((unsigned long long)__double_as_longlong(wq) << 1) != 0ull) I = fma(wq, a.fe_old[(size_t)qq * NI + i], I);
    }
    // Algorithm 2: c_p = dt_p (f*_m - f^E(T^k_{m,p-1})) + I_p; the loop adds dt_p f*_m
    a.cpre[(size_t)(p - 1) * NI + i] = fma(-dtp, a.fe_old[(size_t)(p - 1) * NI + i], I);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Wait until the mbarrier at `bar` completes the phase of parity `parity`,
// for at most `polls` polls; returns false if it gave up. Budgets of fewer than
// 1024 polls test without suspending the thread (mbarrier.test_wait), so that a
// poll is one test; larger budgets use try_wait, which may suspend the thread
// for a while between tests.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long polls) {
    if (polls < 1024) {
        for (long long it = 0; it < polls; ++it) {
            unsigned done;
            asm volatile(
                "{ .reg .pred P1; mbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2; selp.u32 %0, 1, 0, P1; }"
                : "=r"(done)
                : "r"(bar), "r"(parity)
                : "memory");
            if (done) return true;
        }
        return false;
    }
    for (long long it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred P1; mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2; selp.u32 %0, 1, 0, P1; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copies still addressed to a CTA whose exchange wait gave up, by the thread that armed its
// barriers. The CTA sent (and armed the barrier phase of) substeps 1..n_sent and stopped;
// its waits completed up to n_sent - 1. A peer sends the chunk of substep p only after its
// own wait of substep p - 1 completed, which needs this CTA's chunk p - 1; so peers sent this
// CTA chunks of substeps n_sent and n_sent + 1 at most, and `sent` (each CTA's count,
// final once every CTA passed the cluster barrier before this call) says which. The phase of
// substep n_sent was armed for all cs - 1 peers: the bytes of peers that never sent are
// completed here, so that the phase completes exactly when the copies that were sent have
// landed. The phase of substep n_sent + 1 was never armed: it is armed for the copies that
// were sent. Waiting for both phases leaves no copy into this CTA in flight. Returns false if
// a drain wait gave up (an issued copy that never landed).
__device__ bool iface_drain(const int* sent, int rank, int cs, int n_sent, int P, unsigned bytes,
                            const unsigned long long* mbar) {
    auto peers_sent = [&](int p) {
        int k = 0;
        for (int q = 0; q < cs; ++q)
            if (q != rank && *(volatile const int*)(sent + q) >= p) ++k;
        return k;
    };
    // completed phases of barrier b: the substeps 1..n_sent - 1 of parity b
    auto done_phases = [&](int b) { return b == 1 ? n_sent / 2 : (n_sent - 1) / 2; };
    bool ok = true;
    {
        const int b = n_sent & 1;
        const unsigned bar = smem_addr(&mbar[b]);
        const unsigned missing = (unsigned)(cs - 1 - peers_sent(n_sent)) * bytes;
        if (missing)
            asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(missing) : "memory");
        ok = mbar_wait(bar, (unsigned)(done_phases(b) & 1), IFACE_DRAIN_POLLS) && ok;
    }
    if (n_sent + 1 <= P) {
        const int b = (n_sent + 1) & 1;
        const unsigned bar = smem_addr(&mbar[b]);
        const unsigned arriving = (unsigned)peers_sent(n_sent + 1) * bytes;
        if (arriving) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(arriving)
                         : "memory");
            ok = mbar_wait(bar, (unsigned)(done_phases(b) & 1), IFACE_DRAIN_POLLS) && ok;
        }
    }
    return ok;
}

// The P explicit substeps of one interval on the contact DOFs (Algorithm 1 /
// Algorithm 2 inner loops):
//   m T_{m,p} = m T_{m,p-1} + c_p + dt_p f^E(T_{m,p-1}, tau_{m,p-1})
// with c_p from k_iface_prep, on one cluster of CTAs. Every CTA keeps both
// buffers of a full replica of the contact temperatures in shared memory,
// indexed by contact DOF: CTA r owns the contiguous chunk of DOFs
// [r chunk, (r + 1) chunk), so that the loop's per-DOF loads (coupling rows,
// c_p, f*) are coalesced. After a substep's update, lane q of the first warp
// pushes the own chunk into CTA q's replica with a bulk shared-memory copy
// across the cluster that completes a byte count on the receiver's mbarrier;
// waiting for all incoming bytes publishes the substep, so no cluster barrier
// is needed inside the loop. A CTA overwrites a buffer only after it has
// received every peer's next chunk, which each peer sends only after its
// gather from that buffer (program order), so the two buffers suffice.
// Waits are bounded (IfaceArgs::poll_limit). A CTA in which a wait gave up
// stops exchanging (it sends and arms nothing more), reports SDC_ERR_TIMEOUT,
// and before exit drains the copies still addressed to it (iface_drain); a
// closing cluster barrier keeps every CTA resident until all copies from and
// into its shared memory have landed.
//   FP64 (MIX = false): the replica holds T; f^E = cst + sum_k coef_k T_k.
//   Mixed (MIX = true): the replica holds the FP32 deviations T - T_{m-1}
//   (mK over an interval) and f^E = base_p + sum_k coef32_k dT_k, base_p =
//   f^E(T_{m-1}, tau_{m,p}) formed in FP64 by k_iface_prep; each DOF's own T
//   stays FP64.
// Every f^E of the current iterate is stored for the next sweep, and
// ihat = sum_q dt shat_{m,q} f^E_q (its part of I_{m-1}^m) is accumulated.
template <bool MIX, int PER, bool GL, bool STG = false>
__device__ __forceinline__ void iface_loop_impl(const IfaceArgs& a) {
    // one contact DOF per thread leaves registers to prefetch a whole typical row
    constexpr int B = PER == 1 ? (MIX ? 24 : 16) : (PER == 2 ? IFACE_BATCH : 4);
    using V = typename std::conditional<MIX, float, double>::type;
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ __align__(8) unsigned long long mbar[2];
    cg::cluster_group cluster = cg::this_cluster();
    const ContactDev& C = a.C;
    const int NI = C.n_iface;
    const int cs = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int chunk = a.chunk;
    const int P = a.P;
    // [2][cs * chunk]: shared memory, or (GL) global memory for interfaces whose replicas do not
    // fit in shared memory; then owners store their chunk and a cluster barrier publishes it.
    // Staged (GL and a.stage): after that barrier one bulk copy brings the whole replica of the
    // substep into shared memory (one buffer), and the gathers read it there instead of
    // making dependent round trips to L2; the values are the same.
    V* rep = GL ? (V*)a.rep_global : reinterpret_cast<V*>(dyn);
    V* stg = reinterpret_cast<V*>(dyn);
    bool stage_on = GL && STG;
    unsigned stage_issued = 0;  // staged copies issued (one mbarrier phase each, mbar[0])
    const int nthr = (int)blockDim.x;
    // the substep lengths and quadrature weights, formed once (FP64 runs at a small
    // fraction of the FP32 rate, so no thread repeats this work inside the loop)
    __shared__ double s_dtp[MAX_P + 1], s_shat[MAX_P + 1];
    for (int q = threadIdx.x; q < P; q += nthr) {
        const double tn = __dadd_rn(a.st->t0, __dmul_rn((double)a.st->n_done, a.st->dt));
        s_dtp[q + 1] = substep_dt(a, tn, q + 1);
        s_shat[q + 1] = a.Shat[q];
    }

    // Replica position = contact DOF. Shared replicas: CTA r owns the contiguous chunk
    // [r chunk, (r + 1) chunk), which one bulk copy a peer sends. Global replicas (no copies):
    // CTA r owns the 32-DOF tiles r, r + cs, r + 2 cs, ..., so that the DOFs under the
    // moving stock, whose coupling rows are long, spread over all CTAs (chunk is a
    // multiple of 32 there).
    auto owned = [&](int sl) { return GL ? (((sl >> 5) * cs + rank) << 5) + (sl & 31) : rank * chunk + sl; };
    int own[PER];
    double T[PER], T0[PER], fe[PER], mi[PER],
        ih[PER], cn[PER], bn[PER], fs[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int sl = (int)threadIdx.x + nthr * r;
        const int i = owned(sl);
        own[r] = (sl < chunk && i < NI) ? i : -1;
        ih[r] = 0.0;
    }
    // buffer 0 = the replica at tau_{m,0}: T_{m-1} (FP64) or zero deviations (mixed)
    if constexpr (GL) {
        for (int sl = threadIdx.x; sl < chunk; sl += nthr) {
            const int j = owned(sl);
            rep[j] = MIX ? V(0) : (j < NI ? (V)a.Tprev[C.dof[j]] : V(0));
        }
    } else {
        for (int pos = threadIdx.x; pos < cs * chunk; pos += nthr) {
            const int j = pos;
            rep[pos] = MIX ? V(0) : (j < NI ? (V)a.Tprev[C.dof[j]] : V(0));
        }
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[b])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // every CTA has started, filled its replica and initialised its barriers before any copy
    cluster.sync();
    // f^E at tau_{m,0}
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int i = own[r];
        if (i < 0) continue;
        T0[r] = a.Tprev[C.dof[i]];
        T[r] = T0[r];
        mi[r] = C.minv[i];
        double f0;
        if (a.first && a.mode == RHS_PRED) {
            if constexpr (MIX) {
                f0 = a.base[i];
            } else {
                CouplingRowT<B> row;
                coupling_prefetch(a.E, a.slot0, NI, i, row);
                f0 = coupling_apply_shared<B, GL>(a.E, a.slot0, NI, i, row, rep);
            }
        } else {
            f0 = a.first ? a.fe_old[i] : a.fe_prev_end[i];
        }
        fe[r] = f0;
        a.fe_new[i] = f0;
        cn[r] = a.mode == RHS_PRED ? 0.0 : a.cpre[i];
        fs[r] = a.fstar[i];  // f*_m is fixed over the interval
        if constexpr (MIX) bn[r] = a.base[(size_t)NI + i];
    }
    unsigned phase[2] = {0u, 0u};
    const unsigned bytes = (unsigned)(chunk * sizeof(V));
    bool my_to = false;   // this thread's exchange wait gave up
    bool cta_to = false;  // a wait of this CTA gave up: it stopped exchanging after n_sent chunks
    int n_sent = 0;       // substeps whose chunk this CTA sent and whose barrier phase it armed
    for (int p = 1; p <= P; ++p) {
        const int b = p & 1;
        V* buf = rep + (size_t)b * cs * chunk;
        const double dtp = s_dtp[p];
        typename std::conditional<MIX, CouplingRow32T<B>, CouplingRowT<B>>::type row[PER];
        double bp[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int i = own[r];
            if (i < 0) continue;
            if constexpr (MIX) coupling_prefetch32(a.E, a.slot0 + p, NI, i, row[r]);
            else coupling_prefetch(a.E, a.slot0 + p, NI, i, row[r]);
            const double cp = fma(dtp, fs[r], cn[r]);  // c_p (Algorithms 1 and 2)
            bp[r] = bn[r];
            if (p < P) {  // inputs of the next substep, loaded one substep ahead
                cn[r] = a.mode == RHS_PRED ? 0.0 : a.cpre[(size_t)p * NI + i];
                if constexpr (MIX) bn[r] = a.base[(size_t)(p + 1) * NI + i];
            }
            T[r] = fma(fma(dtp, fe[r], cp), mi[r], T[r]);
            buf[i] = MIX ? (V)(T[r] - T0[r]) : (V)T[r];
        }
        if constexpr (GL) {
            cluster.sync();  // the chunks of this substep are in global memory
            if (stage_on) {
                const unsigned sbar = smem_addr(&mbar[0]);
                const unsigned sbytes = (unsigned)((size_t)cs * chunk * sizeof(V));
                if (threadIdx.x == 0) {
                    // the cluster's generic stores to global memory and this CTA's generic reads
                    // of the previous staged replica, ordered before the async-proxy copy
                    asm volatile("fence.proxy.async;" ::: "memory");
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar), "r"(sbytes)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_addr(stg)),
                        "l"(buf), "r"(sbytes), "r"(sbar)
                        : "memory");
                }
                ++stage_issued;
                if (!mbar_wait(sbar, (stage_issued - 1) & 1u, a.poll_limit)) my_to = true;
                // a wait that gave up ends the staging for the whole CTA: no further copy is
                // issued (the step reports SDC_ERR_TIMEOUT), and the outstanding one is drained
                // before exit
                if (__syncthreads_or(my_to)) {
                    stage_on = false;
                    cta_to = true;
                }
            }
        } else {
        // generic-proxy writes of the own chunk become visible to the bulk copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the CTA stops as a whole once a wait of any of its threads gave up
        if (__syncthreads_or(my_to)) {
            cta_to = true;
            break;
        }
        if (threadIdx.x < (unsigned)cs) {  // lane q sends the own chunk to CTA q, all at once
            const int q = (int)threadIdx.x;
            const unsigned src = smem_addr(buf + rank * chunk);
            const unsigned bar = smem_addr(&mbar[b]);
            if (q != rank) {
                unsigned dst, rbar;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(src), "r"(q));
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(bar), "r"(q));
                asm volatile(
                    "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "r"(src), "r"(bytes), "r"(rbar)
                    : "memory");
            }
            if (q == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes * (cs - 1))
                             : "memory");
        }
        n_sent = p;
        if (!mbar_wait(smem_addr(&mbar[b]), phase[b], a.poll_limit)) my_to = true;
        phase[b] ^= 1u;
        }
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int i = own[r];
            if (i < 0) continue;
            // staged: the gathers read the CTA's shared-memory copy of the replica
            constexpr bool FROM_GLOBAL = GL && !STG;
            const V* src = STG ? stg : buf;
            if constexpr (MIX) fe[r] = bp[r] + (double)coupling_apply_shared32<B, FROM_GLOBAL>(a.E, a.slot0 + p, NI, i, row[r], src);
            else fe[r] = coupling_apply_shared<B, FROM_GLOBAL>(a.E, a.slot0 + p, NI, i, row[r], src);
            a.fe_new[(size_t)p * NI + i] = fe[r];
            ih[r] = fma(s_shat[p], fe[r], ih[r]);
        }
    }
    if constexpr (GL) {
        if (cta_to && threadIdx.x == 0) {
            report_status(a.status, SDC_ERR_TIMEOUT);
            // the one staged copy that may still be in flight into this CTA's shared memory
            if (!mbar_wait(smem_addr(&mbar[0]), (stage_issued - 1) & 1u, IFACE_DRAIN_POLLS))
                report_status(a.status, SDC_ERR_TIMEOUT);
        }
        __syncthreads();
    }
    if constexpr (!GL) {
        if (!cta_to) cta_to = __syncthreads_or(my_to);  // a wait of the last substep
        if (cta_to && threadIdx.x == 0) report_status(a.status, SDC_ERR_TIMEOUT);
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int i = own[r];
        if (i < 0) continue;
        a.Tout[C.dof[i]] = T[r];
        if (a.dT) a.dT[C.dof[i]] = (float)(T[r] - T0[r]);
        a.ihat_new[i] = ih[r];
    }
    if constexpr (!GL) {
        if (threadIdx.x == 0) a.sent[rank] = n_sent;
        // every CTA has issued every copy it will issue, and its count in a.sent is visible
        cluster.sync();
        // a CTA whose waits all completed has received every copy addressed to it
        if (cta_to && threadIdx.x == 0 &&
            !iface_drain(a.sent, rank, cs, n_sent, P, bytes, mbar))
            report_status(a.status, SDC_ERR_TIMEOUT);
    }
    // no CTA exits while a bulk copy from or into its shared memory can be in flight
    cluster.sync();
}

// Grid-wide barrier of a cooperative launch (every CTA resident): the CTAs arrive on a
// counter, the last one resets it and advances the generation, the others poll the
// generation, at most `polls` times. Returns false in every thread of a CTA that gave up; the
// kernel goes on (every later wait is bounded too), so every CTA ends, and the step reports
// SDC_ERR_TIMEOUT. Stores before the barrier are visible to loads through L2 after it.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long polls) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;  // the generation cannot advance before this CTA arrives
        int done = 1;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it >= polls) {
                    done = 0;
                    break;
                }
            }
            __threadfence();
        }
        ok = done;
    }
    __syncthreads();
    return ok != 0;
}

// The substeps of iface_loop_impl on a cooperative grid instead of one cluster: one contact
// DOF per thread (DOF = global thread index), as many CTAs as the interface needs, global
// replicas [2][NI] published by the grid barrier. The arithmetic of every DOF is that of the
// cluster forms (same rows, same order), so results are bitwise those of the cluster loop.
// A cluster has at most 16 CTAs; with 27,170 contact DOFs they give a thread four DOFs a
// substep, which this form spreads over about a hundred CTAs.
template <bool MIX>
__device__ __forceinline__ void iface_loop_grid_impl(const IfaceArgs& a) {
    constexpr int B = MIX ? 24 : 16;
    using V = typename std::conditional<MIX, float, double>::type;
    const ContactDev& C = a.C;
    const int NI = C.n_iface;
    const int P = a.P;
    V* rep = (V*)a.rep_global;
    __shared__ double s_dtp[MAX_P + 1], s_shat[MAX_P + 1];
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const double tn = __dadd_rn(a.st->t0, __dmul_rn((double)a.st->n_done, a.st->dt));
        s_dtp[q + 1] = substep_dt(a, tn, q + 1);
        s_shat[q + 1] = a.Shat[q];
    }
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool own = i < NI;
    // buffer 0 = the replica at tau_{m,0}: T_{m-1} (FP64) or zero deviations (mixed)
    if (own) rep[i] = MIX ? V(0) : (V)a.Tprev[C.dof[i]];
    bool ok = grid_barrier(a.gbar, gridDim.x, a.poll_limit);
    double T = 0.0, T0 = 0.0, fe = 0.0, mi = 0.0, ih = 0.0, cn = 0.0, bn = 0.0, fs = 0.0;
    if (own) {
        T0 = a.Tprev[C.dof[i]];
        T = T0;
        mi = C.minv[i];
        double f0;
        if (a.first && a.mode == RHS_PRED) {
            if constexpr (MIX) {
                f0 = a.base[i];
            } else {
                CouplingRowT<B> row;
                coupling_prefetch(a.E, a.slot0, NI, i, row);
                f0 = coupling_apply_shared<B, true>(a.E, a.slot0, NI, i, row, rep);
            }
        } else {
            f0 = a.first ? a.fe_old[i] : a.fe_prev_end[i];
        }
        fe = f0;
        a.fe_new[i] = f0;
        cn = a.mode == RHS_PRED ? 0.0 : a.cpre[i];
        fs = a.fstar[i];
        if constexpr (MIX) bn = a.base[(size_t)NI + i];
    }
    for (int p = 1; p <= P; ++p) {
        V* buf = rep + (size_t)(p & 1) * NI;
        const double dtp = s_dtp[p];
        typename std::conditional<MIX, CouplingRow32T<B>, CouplingRowT<B>>::type row;
        double bp = bn;
        if (own) {
            if constexpr (MIX) coupling_prefetch32(a.E, a.slot0 + p, NI, i, row);
            else coupling_prefetch(a.E, a.slot0 + p, NI, i, row);
            const double cp = fma(dtp, fs, cn);  // c_p (Algorithms 1 and 2)
            if (p < P) {
                cn = a.mode == RHS_PRED ? 0.0 : a.cpre[(size_t)p * NI + i];
                if constexpr (MIX) bn = a.base[(size_t)(p + 1) * NI + i];
            }
            T = fma(fma(dtp, fe, cp), mi, T);
            buf[i] = MIX ? (V)(T - T0) : (V)T;
        }
        ok = grid_barrier(a.gbar, gridDim.x, a.poll_limit) && ok;
        if (own) {
            if constexpr (MIX) fe = bp + (double)coupling_apply_shared32<B, true>(a.E, a.slot0 + p, NI, i, row, buf);
            else fe = coupling_apply_shared<B, true>(a.E, a.slot0 + p, NI, i, row, buf);
            a.fe_new[(size_t)p * NI + i] = fe;
            ih = fma(s_shat[p], fe, ih);
        }
    }
    if (!ok && threadIdx.x == 0) report_status(a.status, SDC_ERR_TIMEOUT);
    if (own) {
        a.Tout[C.dof[i]] = T;
        if (a.dT) a.dT[C.dof[i]] = (float)(T - T0);
        a.ihat_new[i] = ih;
    }
}

__global__ void __launch_bounds__(IFACE_GRID_THREADS) k_iface_loop_grid(IfaceArgs a) { iface_loop_grid_impl<false>(a); }
__global__ void __launch_bounds__(IFACE_GRID_THREADS) k_iface_loop_mx_grid(IfaceArgs a) { iface_loop_grid_impl<true>(a); }

// shared-memory replicas with one (chunk <= IFACE_THREADS) or two contact DOFs per thread;
// global replicas with up to four (interfaces too large for shared memory)
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop1(IfaceArgs a) { iface_loop_impl<false, 1, false>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop(IfaceArgs a) { iface_loop_impl<false, 2, false>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_gl(IfaceArgs a) { iface_loop_impl<false, 4, true>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_mx1(IfaceArgs a) { iface_loop_impl<true, 1, false>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_mx(IfaceArgs a) { iface_loop_impl<true, 2, false>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_mx_gl(IfaceArgs a) { iface_loop_impl<true, 4, true>(a); }
// global replicas staged in shared memory after every substep (one buffer of cs x chunk values)
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_gls(IfaceArgs a) { iface_loop_impl<false, 4, true, true>(a); }
__global__ void __launch_bounds__(IFACE_THREADS) k_iface_loop_mx_gls(IfaceArgs a) { iface_loop_impl<true, 4, true, true>(a); }

// ------------------------------------------------------------------ diagnostics

// r^k = max_m || m T_m - m T_n - sum_{j<=m} I_{j-1}^j ||_inf (Eq. residual)
__global__ void k_residual(ResidualArgs a) {
    double v[1] = {0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
            const double m = a.mass[i];
            const double tn = a.Tn[i];
            const int pa = a.pos[i];
            double cum = 0.0, r = 0.0;
            for (int mm = 0; mm < a.M; ++mm) {
                double I = 0.0;
                for (int j = 0; j < a.M; ++j) I = fma(a.Sdt[mm][j], a.FI[j][i], I);
                if (pa >= 0 && a.ihat[mm]) I += a.ihat[mm][pa];
                cum += I;
                r = fmax(r, fabs(m * a.Tm[mm][i] - m * tn - cum));
            }
            v[0] = fmax(v[0], r);
    }
    double out[1];
    if (reduce_last<1, true>(v, a.partials, a.counter, out) && threadIdx.x == 0) *a.out = out[0];
}

// heat[0] = sum over stand rows of m T, heat[1] = stock rows
__global__ void k_heat(const double* __restrict__ mass, const double* __restrict__ T, int64_t n, int64_t n_fix,
                       double* partials, unsigned int* counter, double* heat) {
    double v[2] = {0.0, 0.0};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
            const double h = mass[i] * T[i];
            if (i < n_fix) v[0] += h; else v[1] += h;
    }
    double out[2];
    if (reduce_last<2, false>(v, partials, counter, out) && threadIdx.x == 0) {
        heat[0] = out[0];
        heat[1] = out[1];
    }
}

// friction energy of the step: sum over intervals and contact DOFs of ihat
// (exchange terms cancel between the bodies); then advance the step counter.
__global__ void k_step_end(StepState* st, const double* ihat, int n_int, int NI) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int m = 0; m < n_int; ++m)
        for (int i = threadIdx.x; i < NI; i += blockDim.x) acc += ihat[(size_t)m * NI + i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        st->friction_in += t;
        st->n_done += 1;
    }
}

}  // namespace sdc
