// One sketched-GMRES cycle on the device for every problem of a batch (Section 3; Eq. 3 with r0 = v_j and zero
// initial guess).
//
// Storage: the basis vectors are kept unnormalised, b_l = sigma_l u_l; scale factors live in scalars and a stored
// vector is only ever rescaled by a power of two.  Per inner step i (0-based; the paper's i+1):
//   k_inner_spmv  w' = A u_i, the truncated-Arnoldi dot products u_l^T w' for the last t basis vectors
//                 (Section 4.1), ||u_i||^2, and the per-block partial sketch S w' -- one pass over A; the row block of
//                 w' stays in shared memory for the sketch gather lists.  In FP64 the sketch partials are accumulated
//                 exactly in 64-bit fixed point (integer adds), which keeps the scarce FP64 pipe for the SpMV.
//   k_inner_axpy  sigma_i = 1/||u_i||, h_l = b_l^T A b_i, the sketched column S A b_i = sigma_i S w', and the next
//                 stored vector u_{i+1} = 2^p_i (w' - sum_l sigma_l^2 (u_l^T w') u_l), with 2^p_i the power of two
//                 just below sigma_i (an exact rescaling that keeps stored norms O(||A||) instead of growing like
//                 ||A||^i).
//   k_inner_qr    per problem a cluster of CTAs: Gram-Schmidt with one reorthogonalisation pass of S A b_i against Q
//                 (Section 3, C2), the condition proxy max|r_ll|/min|r_ll| (rule C2), the running sketched residual
//                 (rule C3) and C1.  It runs on a second stream, overlapping the next step's SpMV; a step that runs
//                 past the end of a problem's cycle is discarded.
// After the cycle: k_inner_ls solves R_k y = (Q^T S v)_k and k_inner_gemv forms z_j = B_k y_k (FP64 output).
// The step kernels (k_inner_spmv, k_inner_axpy and the fused k_inner_step) live in inner_step.cuh and are
// instantiated per precision in inner_f64.cu, inner_f32.cu and inner_bf16.cu; this file holds the QR, the least
// squares, z, the cycle reset and the launchers.
#include "inner_step.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace sfg {

// ---------------------------------------------------------------------------------------------------------------
// Sketched QR update of column i, one cluster of nq CTAs per problem (cluster index = problem); CTA q owns rows [s q / nq, s (q+1) / nq) of Q and of the working vectors.  Q is kept twice: column-major
// (Q[l*s + r]) for the projection Q^T p, where each thread takes a column and streams its rows, and row-major
// (Qt[r*m + l]) for the subtraction p -= Q a, where each thread takes a row and streams its columns: every lane reads
// contiguous memory, so each load instruction keeps 32 cache lines in flight and each line serves 16 elements (the
// update is bound by the latency of these reads, not by their bandwidth).  When the CTA has few columns to project
// (small i) or few rows (s / nq below 128), the work is split further: the projection's rows into up to 8 groups,
// the subtraction's columns into up to 4, with the group partials combined in group order.  Partial dot products of
// the CTAs go through distributed shared memory and are summed in rank order (deterministic, the same values in
// every CTA, so every decision is taken identically everywhere).  Five cluster barriers per update: one per
// Gram-Schmidt pass (the two passes' partials live in separate buffers), one for ||p||^2 and p^T e together
// (d_i = p^T e / r_ii), one for the updated residual norm, and a last one before any CTA leaves.  Each CTA reads the
// stop state itself (written by earlier launches; the one field another stream may change meanwhile, the breakdown
// step, only ever moves to values above i).  CTAs are small (128 threads, at most 56 registers) so they fit beside
// the inner step's CTAs.
__device__ __forceinline__ double qr_rank_sum(cg::cluster_group& cl, double* base, int off, int nq) {
    double acc = 0.0;
#pragma unroll 8
    for (int r2 = 0; r2 < nq; ++r2) acc += cl.map_shared_rank(base, r2)[off];
    return acc;
}

// Sum over the CTA's 128 threads of v (warp trees, then the 4 warps in order); valid in thread 0 (0 elsewhere).
__device__ __forceinline__ double qr_block_sum(double v, double* red4) {
    v = warp_sum(v);
    __syncthreads();  // red4 is free (its previous values have been read)
    if ((threadIdx.x & 31) == 0) red4[threadIdx.x >> 5] = v;
    __syncthreads();
    return (threadIdx.x == 0) ? (red4[0] + red4[1]) + (red4[2] + red4[3]) : 0.0;
}

// Sum of x[u] * y[u] for u in [0, cnt), x contiguous (each lane of a warp streams its own stretch of Q, so every load
// instruction has 32 cache lines in flight and every line serves 16 consecutive elements from L1): chunks of eight
// loads, with the lane's lines four ahead prefetched into L1 (no registers held for them); four accumulators,
// combined in a fixed order.
__device__ __forceinline__ double qr_dot(const double* __restrict__ x, const double* __restrict__ y, int cnt) {
    for (int k = 0; k < 64 && k < cnt; k += 16) prefetch_l1(x + k);
    double c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = 0.0;
    int k = 0;
    for (; k + 8 <= cnt; k += 8) {
        if ((k & 15) == 0 && k + 64 < cnt) prefetch_l1(x + k + 64);
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = x[k + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u & 3] = fma(v[u], y[k + u], c[u & 3]);
    }
    for (; k < cnt; ++k) c[0] = fma(x[k], y[k], c[0]);  // at most 7, from lines already in L1
    return (c[0] + c[1]) + (c[2] + c[3]);
}

constexpr int kQrThreads = 128;

__global__ void __launch_bounds__(kQrThreads, 9) k_inner_qr(const Plan P, int i) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank(), nq = (int)cl.num_blocks();
    const int prob = blockIdx.x / nq;
    const int s = P.s, m = P.m;
    const double* __restrict__ C = P.C + (int64_t)prob * m * s;
    double* __restrict__ Q = P.Q + (int64_t)prob * m * s;
    double* __restrict__ Qt = P.Qt + (int64_t)prob * m * s;
    double* __restrict__ R = P.R + (int64_t)prob * m * m;
    double* __restrict__ d = P.d + (int64_t)prob * m;
    double* __restrict__ e = P.e + (int64_t)prob * s;
    double* __restrict__ rho = P.rho + (int64_t)prob * m;
    CycleState* cyc = P.cyc + prob;
    const int rlo = (int)((int64_t)s * q / nq), rhi = (int)((int64_t)s * (q + 1) / nq), nr = rhi - rlo;
    const int nrmax = (s + nq - 1) / nq;
    extern __shared__ double qsm[];
    double* p = qsm;               // [nrmax] this CTA's rows of the working vector
    double* apart = qsm + nrmax;   // [2][m] partial projections over this CTA's rows, one buffer per pass
    double* a = apart + 2 * m;     // [m] full projections
    __shared__ double red4[4];
    __shared__ double scal[4];
    __shared__ double bc[4];            // scalars formed by thread 0 for the CTA (FP64 division and square roots
                                        // cost tens of FP64-pipe cycles per warp: once per CTA, not per thread)
    __shared__ double grp[kQrThreads];  // group partials of a split projection or subtraction
    const int tid = threadIdx.x;
    // the cycle state as earlier launches left it (the same for every CTA of the cluster)
    const double dmax0 = cyc->dmax, dmin0 = cyc->dmin, thr = cyc->cond_thr;
    const int code = (cyc->stopped || (P.pflag[prob] & 1)) ? 1 : (cyc->brk_step <= i ? 2 : 0);
    if (code) {
        if (code == 2 && q == 0 && tid == 0) {
            cyc->stopped = 1;  // u_i has zero (or non-finite) norm: the cycle keeps k = i columns
            cyc->reason = cyc->brk_reason;
        }
        return;  // the whole cluster returns
    }
    for (int r = tid; r < nr; r += kQrThreads) p[r] = C[(int64_t)i * s + rlo + r];
    // projection split: Gp groups of rows (Gp * i <= 128 threads), Wp threads per group over the columns
    int Gp = 1;
    while (Gp < 8 && 2 * Gp * i <= kQrThreads && 2 * Gp * 8 <= nr) Gp *= 2;
    const int Wp = kQrThreads / Gp, gp = tid / Wp, wp = tid % Wp;
    const int pr0 = nr * gp / Gp, pr1 = nr * (gp + 1) / Gp;
    // subtraction split: Wr threads over the rows (a power of two from 32 to 128, so that Gs Wr = 128 and every
    // thread has a group), Gs groups of columns
    int Wr = 32;
    while (Wr < nr && Wr < kQrThreads) Wr *= 2;
    const int Gs = kQrThreads / Wr, gs = tid / Wr, ws = tid % Wr;
    const int sl0 = i * gs / Gs, sl1 = i * (gs + 1) / Gs;
    const unsigned long long keep = l2_keep_policy();  // Q and Qt are read again at every update of the cycle
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        double* ap = apart + pass * m;
        // this CTA's part of Q^T p: column l by thread wp of group gp, over the group's rows (contiguous in Q)
        for (int l = wp; l < i; l += Wp) {
            const double v = qr_dot(Q + (int64_t)l * s + rlo + pr0, p + pr0, pr1 - pr0);
            if (Gp == 1) ap[l] = v;
            else grp[gp * i + l] = v;
        }
        if (Gp > 1) {
            __syncthreads();
            for (int l = tid; l < i; l += kQrThreads) {
                double v = 0.0;
                for (int g = 0; g < Gp; ++g) v += grp[g * i + l];
                ap[l] = v;
            }
        }
        cl.sync();  // this pass's partials of every CTA are in place
        for (int l = tid; l < i; l += kQrThreads) a[l] = qr_rank_sum(cl, ap, l, nq);
        __syncthreads();
        // p -= Q a over this CTA's rows: row r by thread ws, the columns of group gs (contiguous in Qt)
        for (int r = ws; r < nr; r += Wr) {
            const double v = qr_dot(Qt + (int64_t)(rlo + r) * m + sl0, a + sl0, sl1 - sl0);
            if (Gs == 1) p[r] -= v;
            else grp[gs * Wr + r] = v;
        }
        if (Gs > 1) {
            __syncthreads();
            for (int r = tid; r < nr; r += kQrThreads) {
                double v = 0.0;
                for (int g = 0; g < Gs; ++g) v += grp[g * Wr + r];
                p[r] -= v;
            }
        }
        if (q == 0)
            for (int l = tid; l < i; l += kQrThreads) R[(int64_t)i * m + l] = (pass ? R[(int64_t)i * m + l] : 0.0) + a[l];
        __syncthreads();
    }
    // r_ii = ||p|| and p^T e from one exchange
    double v2 = 0.0, pe = 0.0;
    for (int r = tid; r < nr; r += kQrThreads) {
        v2 += p[r] * p[r];
        pe += p[r] * e[rlo + r];
    }
    v2 = qr_block_sum(v2, red4);
    pe = qr_block_sum(pe, red4);
    if (tid == 0) {
        scal[0] = v2;
        scal[1] = pe;
    }
    cl.sync();
    if (tid == 0) {
        const double rii0 = sqrt(qr_rank_sum(cl, scal, 0, nq));
        const double dmx = fmax(dmax0, rii0);
        const double dmn = (i == 0) ? rii0 : fmin(dmin0, rii0);
        bc[0] = rii0;
        bc[1] = qr_rank_sum(cl, scal, 1, nq);
        bc[2] = (dmn > 0.0) ? dmx / dmn : INFINITY;  // the condition proxy
        bc[3] = 1.0 / rii0;
    }
    __syncthreads();
    const double rii = bc[0], pet = bc[1], kappa = bc[2], inv = bc[3];
    const double dmax = fmax(dmax0, rii);
    const double dmin = (i == 0) ? rii : fmin(dmin0, rii);
    if (!(kappa <= thr)) {  // C2 (also rii == 0 or NaN): drop column i, keep k = i
        if (q == 0 && tid == 0) {
            cyc->stopped = 1;
            cyc->k = i;
            cyc->reason = (i == 0) ? 5 : 2;
        }
        cl.sync();  // no CTA leaves while another may still read its shared memory
        return;
    }
    const double di = pet * inv;
    double ee = 0.0;
    for (int r = tid; r < nr; r += kQrThreads) {
        const double qv = p[r] * inv;
        st_keep(Q + (int64_t)i * s + rlo + r, qv, keep);
        st_keep(Qt + (int64_t)(rlo + r) * m + i, qv, keep);
        const double ev = e[rlo + r] - di * qv;
        e[rlo + r] = ev;
        ee += ev * ev;
    }
    ee = qr_block_sum(ee, red4);
    if (tid == 0) scal[2] = ee;
    cl.sync();
    if (q == 0 && tid == 0) {
        const double rh = sqrt(qr_rank_sum(cl, scal, 2, nq));
        R[(int64_t)i * m + i] = rii;
        d[i] = di;
        rho[i] = rh;
        cyc->dmax = dmax;
        cyc->dmin = dmin;
        cyc->k = i + 1;
        cyc->rho = rh;
        if (cyc->c3_on && cyc->c3_scale * rh <= cyc->c3_tol) {
            cyc->stopped = 1;
            cyc->reason = 3;
        } else if (i + 1 == m) {
            cyc->stopped = 1;
            cyc->reason = 1;
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------------------------------------------
// The same sketched QR update for small sketches (qr_small_fits, few problems), one CTA of kQrSmallThreads
// threads per problem and no cluster.  An update of a small sketch is a chain of dependent steps whose cost is the
// number of round trips to memory, so every global input -- the columns 0..i-1 of Q, the new column of C, the
// residual sketch e, the cycle state -- is loaded into shared memory in one wave of loads at the start, and the two
// Gram-Schmidt passes, the norms and the stop tests then run on shared memory (block barriers instead of cluster
// barriers and distributed-shared-memory exchanges).  Projections: warp w takes columns w, w + 16, ..., its lanes
// strided over the rows, then the warp's shuffle tree.  Subtraction: G threads per row (G s <= the CTA), each over a
// contiguous share of the columns, the G partials added by a shuffle tree.  Block sums: warp trees, then the warps
// in order.  Only Q is written (not its row-major copy Qt, which only the cluster kernel reads).  The decisions
// (rules C1-C3, the breakdown and C2 stops) are those of k_inner_qr.
constexpr int kQrSmallThreads = 512;

// Sum of v over the threads of the first nws warps (the others hold no rows): warp trees, then the warps in order;
// valid in thread 0 (0 elsewhere).  FP64 arithmetic is scarce on this GPU, so no thread adds what it does not need.
__device__ __forceinline__ double qr_small_sum(double v, double* red, int nws) {
    const int warp = threadIdx.x >> 5;
    if (warp < nws) v = warp_sum(v);
    __syncthreads();  // red is free (its previous values have been read)
    if (warp < nws && (threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nws; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(kQrSmallThreads) k_inner_qr_small(const Plan P, int i) {
    constexpr int nw = kQrSmallThreads / 32;
    const int prob = blockIdx.x;
    const int s = P.s, m = P.m;
    const double* __restrict__ C = P.C + (int64_t)prob * m * s;
    double* __restrict__ Q = P.Q + (int64_t)prob * m * s;
    double* __restrict__ R = P.R + (int64_t)prob * m * m;
    double* __restrict__ d = P.d + (int64_t)prob * m;
    double* __restrict__ e = P.e + (int64_t)prob * s;
    double* __restrict__ rho = P.rho + (int64_t)prob * m;
    CycleState* cyc = P.cyc + prob;
    extern __shared__ double qsm[];
    double* qs = qsm;              // [i s] columns 0..i-1 of Q (column-major)
    double* p = qs + (int64_t)i * s;  // [s] the working vector
    double* es = p + s;            // [s] e
    double* a1 = es + s;           // [m] first-pass projections
    double* a = a1 + m;            // [m] projections of the current pass
    __shared__ double red[nw];
    __shared__ double cst[3];
    __shared__ double bc[4];  // scalars formed by thread 0 (one square root and divisions per update, not per thread)
    __shared__ int code_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        cst[0] = cyc->dmax;
        cst[1] = cyc->dmin;
        cst[2] = cyc->cond_thr;
        code_sh = (cyc->stopped || (P.pflag[prob] & 1)) ? 1 : (cyc->brk_step <= i ? 2 : 0);
    }
    const int nq = i * s;
    for (int k = tid; k < nq; k += kQrSmallThreads) qs[k] = Q[k];
    for (int r = tid; r < s; r += kQrSmallThreads) {
        p[r] = C[(int64_t)i * s + r];
        es[r] = e[r];
    }
    __syncthreads();
    const int code = code_sh;
    if (code) {
        if (code == 2 && tid == 0) {
            cyc->stopped = 1;  // u_i has zero (or non-finite) norm: the cycle keeps k = i columns
            cyc->reason = cyc->brk_reason;
        }
        return;
    }
    int G = 1;
    while (G < 32 && 2 * G * s <= kQrSmallThreads) G *= 2;
    const int rg = tid / G, gg = tid % G;
    const int c0 = i * gg / G, c1 = i * (gg + 1) / G;
    for (int pass = 0; pass < 2; ++pass) {
        // a = Q^T p: column l by warp l % nw
        for (int l = warp; l < i; l += nw) {
            const double* ql = qs + (int64_t)l * s;
            double acc = 0.0;
            for (int r = lane; r < s; r += 32) acc = fma(ql[r], p[r], acc);
            acc = warp_sum(acc);
            if (lane == 0) a[l] = acc;
        }
        __syncthreads();
        // p -= Q a: row r by its G threads
        for (int base = 0; base < s; base += kQrSmallThreads / G) {  // the same trip count in every thread
            const int r = base + rg;
            double acc = 0.0;
            if (r < s)
                for (int l = c0; l < c1; ++l) acc = fma(qs[(int64_t)l * s + r], a[l], acc);
            for (int o = 1; o < G; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);  // all lanes take part
            if (r < s && gg == 0) p[r] -= acc;
        }
        if (pass == 0)
            for (int l = tid; l < i; l += kQrSmallThreads) a1[l] = a[l];
        __syncthreads();
    }
    for (int l = tid; l < i; l += kQrSmallThreads) R[(int64_t)i * m + l] = a1[l] + a[l];
    // r_ii = ||p|| and p^T e
    const int nws = (min(s, kQrSmallThreads) + 31) / 32;  // warps that hold rows
    double v2 = 0.0, pe = 0.0;
    for (int r = tid; r < s; r += kQrSmallThreads) {
        v2 = fma(p[r], p[r], v2);
        pe = fma(p[r], es[r], pe);
    }
    v2 = qr_small_sum(v2, red, nws);
    pe = qr_small_sum(pe, red, nws);
    if (tid == 0) {
        const double rii0 = sqrt(v2);
        const double dmx = fmax(cst[0], rii0);
        const double dmn = (i == 0) ? rii0 : fmin(cst[1], rii0);
        bc[0] = rii0;
        bc[1] = pe;
        bc[2] = (dmn > 0.0) ? dmx / dmn : INFINITY;  // the condition proxy
        bc[3] = 1.0 / rii0;
    }
    __syncthreads();
    const double rii = bc[0], pet = bc[1], kappa = bc[2], inv = bc[3];
    const double dmax = fmax(cst[0], rii);
    const double dmin = (i == 0) ? rii : fmin(cst[1], rii);
    if (!(kappa <= cst[2])) {  // C2 (also rii == 0 or NaN): drop column i, keep k = i
        if (tid == 0) {
            cyc->stopped = 1;
            cyc->k = i;
            cyc->reason = (i == 0) ? 5 : 2;
        }
        return;
    }
    const double di = pet * inv;
    double ee = 0.0;
    for (int r = tid; r < s; r += kQrSmallThreads) {
        const double qv = p[r] * inv;
        Q[(int64_t)i * s + r] = qv;
        const double ev = es[r] - di * qv;
        e[r] = ev;
        ee = fma(ev, ev, ee);
    }
    ee = qr_small_sum(ee, red, nws);
    if (tid == 0) {
        const double rh = sqrt(ee);
        R[(int64_t)i * m + i] = rii;
        d[i] = di;
        rho[i] = rh;
        cyc->dmax = dmax;
        cyc->dmin = dmin;
        cyc->k = i + 1;
        cyc->rho = rh;
        if (cyc->c3_on && cyc->c3_scale * rh <= cyc->c3_tol) {
            cyc->stopped = 1;
            cyc->reason = 3;
        } else if (i + 1 == m) {
            cyc->stopped = 1;
            cyc->reason = 1;
        }
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Per problem (one CTA of 128 threads): y = R_k^{-1} d by column-oriented back substitution, coef_l = y_l sigma_l.
// Step l divides by r_ll and subtracts y_l times column l of R from the rows above it, one row per thread; the next
// column is loaded while the current one is applied, so each step costs a barrier rather than an L2 round trip.
constexpr int kLsThreads = 128;
__global__ void __launch_bounds__(kLsThreads) k_inner_ls(const Plan P) {
    extern __shared__ double rhs[];  // [k]
    __shared__ double yl_sh;
    const int p = blockIdx.x, m = P.m;
    if (P.pflag[p] & 1) return;
    const double* R = P.R + (int64_t)p * m * m;  // column-major: R[l*m + q] = R_{q,l}
    const double* d = P.d + (int64_t)p * m;
    const double* sigma = P.sigma + (int64_t)p * (m + 1);
    double* y = P.y + (int64_t)p * m;
    double* coef = P.coef + (int64_t)p * m;
    const int k = P.cyc[p].k;
    if (k <= 32) {
        // one warp: lane q holds row q of the right-hand side, its row of R (one load wave) and 1 / r_qq (the
        // divisions of all rows at once); step l forms y_l = rhs_l (1 / r_ll) in lane l, shuffles it to the other
        // lanes, and the rows above l subtract r_ql y_l in parallel -- warp shuffles instead of block barriers and one
        // FP64 multiply-add per step on the critical path
        if (threadIdx.x >= 32) return;
        const int q = threadIdx.x;
        double r = (q < k) ? d[q] : 0.0;
        double rq[32];
#pragma unroll
        for (int l = 0; l < 32; ++l) rq[l] = (l < k && q <= l) ? R[(int64_t)l * m + q] : 0.0;
        double rqq = 1.0;
#pragma unroll
        for (int l = 0; l < 32; ++l)
            if (l == q && q < k) rqq = rq[l];
        const double inv = 1.0 / rqq;
        for (int l = k - 1; l >= 0; --l) {
            double rql = 0.0;  // r_ql of this lane's row
#pragma unroll
            for (int u = 0; u < 32; ++u)
                if (u == l) rql = rq[u];
            const double yl = __shfl_sync(0xffffffffu, r * inv, l);
            if (q < l) r = fma(-rql, yl, r);
            if (q == l) {
                y[l] = yl;
                coef[l] = yl * sigma[l];
            }
        }
        return;
    }
    for (int l = threadIdx.x; l < k; l += kLsThreads) rhs[l] = d[l];
    // this thread's rows q = threadIdx.x + 128 j; its entries of the current column l are loaded one column ahead
    constexpr int kRows = kMaxM / kLsThreads;
    double col[kRows];
    auto load_col = [&](int l) {
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const int q = threadIdx.x + kLsThreads * j;
            col[j] = (l >= 0 && q <= l) ? R[(int64_t)l * m + q] : 0.0;
        }
    };
    load_col(k - 1);
    __syncthreads();
    for (int l = k - 1; l >= 0; --l) {
        if (threadIdx.x == (l % kLsThreads)) {
            double rll = 0.0;
#pragma unroll
            for (int j = 0; j < kRows; ++j)
                if (threadIdx.x + kLsThreads * j == l) rll = col[j];
            const double yl = rhs[l] / rll;
            yl_sh = yl;
            y[l] = yl;
            coef[l] = yl * sigma[l];
        }
        double cur[kRows];
#pragma unroll
        for (int j = 0; j < kRows; ++j) cur[j] = col[j];
        load_col(l - 1);
        __syncthreads();  // y_l is in yl_sh
        const double yl = yl_sh;
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const int q = threadIdx.x + kLsThreads * j;
            if (q < l) rhs[q] -= cur[j] * yl;
        }
        __syncthreads();  // rhs[l - 1] is final before its owner divides; yl_sh is free again
    }
}

// z = sum_{l<k} coef_l u_l over each block's rows, FP64 output.  FP64 basis: FP64 FMAs.  FP32/BF16 basis: the FP64
// coefficients are split into two FP32 parts and the sum is carried as an unevaluated FP32 pair (TwoSum, and FMA
// for the exact product error), close to FP64 accuracy on the FP32 pipe.
template <typename VT>
__global__ void __launch_bounds__(256) k_inner_gemv(const Plan P, double* __restrict__ z) {
    __shared__ double cf[kMaxM];
    __shared__ float ch[kMaxM], clo[kMaxM];
    const BlockInfo bi = block_info(P, blockIdx.x);
    const int p = bi.prob;
    if (P.pflag[p] & 1) return;
    const int k = P.cyc[p].k, N = P.N;
    const VT* Ub = (const VT*)P.U;
    const double* coef = P.coef + (int64_t)p * P.m;
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        const double c = coef[l];
        cf[l] = c;
        const float hi = (float)c;
        ch[l] = hi;
        clo[l] = (float)(c - (double)hi);
    }
    __syncthreads();
    for (int kk = threadIdx.x; kk < bi.len; kk += blockDim.x) {
        const int64_t r = bi.v0 + kk;
        if constexpr (sizeof(VT) == 8) {
            double acc = 0.0;
            for (int l = 0; l < k; ++l) acc += cf[l] * (double)ld_plain(Ub + (int64_t)l * N + r);
            z[r] = acc;
        } else {
            float sh = 0.f, sl = 0.f;
            for (int l = 0; l < k; ++l) {
                const float u = ld_plain(Ub + (int64_t)l * N + r);
                const float pr = ch[l] * u;
                const float pe = fmaf(ch[l], u, -pr) + clo[l] * u;  // exact product error + low-part term
                const float t1 = sh + pr;                            // TwoSum(sh, pr)
                const float bv = t1 - sh;
                const float err = (sh - (t1 - bv)) + (pr - bv);
                sh = t1;
                sl += err + pe;
            }
            z[r] = (double)sh + (double)sl;
        }
    }
}

template <typename VT>
__global__ void k_export_basis(const Plan P, int count, double* __restrict__ out) {
    const BlockInfo bi = block_info(P, blockIdx.x);
    const double* sigma = P.sigma + (int64_t)bi.prob * (P.m + 1);
    const VT* Ub = (const VT*)P.U;
    for (int kk = threadIdx.x; kk < bi.len; kk += blockDim.x) {
        const int64_t r = bi.v0 + kk;
        for (int l = 0; l < count; ++l)
            out[(int64_t)l * P.N + r] = sigma[l] * (double)ld_plain(Ub + (int64_t)l * P.N + r);
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Start of inner cycle j, per problem: reset the cycle state (C3 scale = FFOM residual of the previous outer step,
// beta at the first, Eq. 5); a problem that is done is marked stopped so every inner kernel skips it.
__global__ void k_cycle_reset(const Plan P, int j, int c3_on, double cond_thr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.P) return;
    CycleState* cyc = P.cyc + p;
    cyc->stopped = (P.pflag[p] & 1) ? 1 : 0;
    cyc->k = 0;
    cyc->reason = 0;
    cyc->brk_step = INT_MAX;
    cyc->brk_reason = 0;
    cyc->dmax = 0.0;
    cyc->dmin = INFINITY;
    cyc->rho = INFINITY;
    cyc->cond_thr = cond_thr;
    if (p == 0 && P.gsync) {  // the fused step's grid counters (0: phase-1 partials, 2: sketch partials), give-up flag
        P.gsync[0] = 0;
        P.gsync[1] = 0;
        P.gsync[2] = 0;
    }
    if (j >= 0) {
        const OuterState* ost = P.ost + p;
        const double sc = (j == 0) ? ost->beta : ost->ffom;
        cyc->c3_scale = sc;
        cyc->c3_tol = ost->tol_abs;
        cyc->c3_on = (c3_on && isfinite(sc)) ? 1 : 0;
    } else {
        cyc->c3_scale = INFINITY;
        cyc->c3_tol = 0.0;
        cyc->c3_on = 0;
    }
    P.sigma[(int64_t)p * (P.m + 1)] = 1.0;
}

void launch_cycle_start(const Plan& p, int j, const double* v, const double* vscale, int vstride, int c3_on,
                        double cond_thr) {
    k_cycle_reset<<<(p.P + 127) / 128, 128, 0, p.st>>>(p, j, c3_on, cond_thr);
    launch_sketch_partials(p, v, vscale, vstride, p.U, p.cpart);
    launch_sketch_reduce(p, p.cpart, p.c0, p.e);
    ++g_launches;
}

void launch_inner_spmv(const Plan& p, int i) {
    if (p.prec == kFP64) inner_spmv_f64(p, i);
    else if (p.prec == kFP32) inner_spmv_f32(p, i);
    else inner_spmv_bf16(p, i);
    ++g_launches;
}

bool launch_inner_step(const Plan& p, int i, bool last) {
    if (!p.gsync) return false;
    bool ok;
    if (p.prec == kFP64) ok = inner_step_f64(p, i, last);
    else if (p.prec == kFP32) ok = inner_step_f32(p, i, last);
    else ok = inner_step_bf16(p, i, last);
    if (ok) ++g_launches;
    return ok;
}

void launch_inner_axpy(const Plan& p, int i, bool last) {
    if (p.prec == kFP64) inner_axpy_f64(p, i, last);
    else if (p.prec == kFP32) inner_axpy_f32(p, i, last);
    else inner_axpy_bf16(p, i, last);
    ++g_launches;
}

cudaError_t launch_inner_qr(const Plan& p, int i, cudaStream_t st) {
    if (p.qr_cluster == 0) {  // small sketch: one CTA per problem, Q's columns 0..i-1 in shared memory
        const size_t sm = ((size_t)i * p.s + 2 * (size_t)p.s + 2 * (size_t)p.m) * sizeof(double);
        set_smem((const void*)k_inner_qr_small, sm);
        k_inner_qr_small<<<p.P, kQrSmallThreads, sm, st>>>(p, i);
        ++g_launches;
        return cudaGetLastError();
    }
    const int nq = p.qr_cluster;
    const int nrmax = (p.s + nq - 1) / nq;
    const size_t sm = (size_t)(nrmax + 3 * p.m) * sizeof(double);
    set_smem((const void*)k_inner_qr, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nq * p.P), 1, 1);
    cfg.blockDim = dim3(kQrThreads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nq;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++g_launches;
    return cudaLaunchKernelEx(&cfg, k_inner_qr, p, i);
}

void launch_inner_finish(const Plan& p, double* z) {
    set_smem((const void*)k_inner_ls, (size_t)p.m * sizeof(double));
    k_inner_ls<<<p.P, kLsThreads, (size_t)p.m * sizeof(double), p.st>>>(p);
    if (p.prec == kFP64) k_inner_gemv<double><<<p.nblk, 256, 0, p.st>>>(p, z);
    else if (p.prec == kFP32) k_inner_gemv<float><<<p.nblk, 256, 0, p.st>>>(p, z);
    else k_inner_gemv<__nv_bfloat16><<<p.nblk, 256, 0, p.st>>>(p, z);
    g_launches += 2;
}

void launch_export_basis(const Plan& p, double* out, int count) {
    if (p.prec == kFP64) k_export_basis<double><<<p.nblk, 256, 0, p.st>>>(p, count, out);
    else if (p.prec == kFP32) k_export_basis<float><<<p.nblk, 256, 0, p.st>>>(p, count, out);
    else k_export_basis<__nv_bfloat16><<<p.nblk, 256, 0, p.st>>>(p, count, out);
    ++g_launches;
}

}  // namespace sfg
