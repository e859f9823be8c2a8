// One sketched-GMRES cycle on the device (Section 3; Eq. 3 with r0 = v_j and zero initial guess).
//
// Storage: the basis vectors are kept unnormalised, b_l = sigma_l u_l; scale factors live in scalars and a stored
// vector is only ever rescaled by a power of two.  Per inner step i (0-based; the paper's i+1):
//   k_inner_spmv  w' = A u_i, the truncated-Arnoldi dot products u_l^T w' for the last t basis vectors
//                 (Section 4.1), and the per-block partial sketch S w' -- one pass over A; the row block of w' stays
//                 in shared memory for the sketch gather lists.  In FP64 the sketch partials are accumulated exactly
//                 in 64-bit fixed point (integer adds), which keeps the scarce FP64 pipe for the SpMV.
//   k_inner_axpy  sigma_i = 1/||u_i||, h_l = b_l^T A b_i, the sketched column S A b_i = sigma_i S w', and the next
//                 stored vector u_{i+1} = 2^p_i (w' - sum_l sigma_l^2 (u_l^T w') u_l), with 2^p_i the power of two
//                 nearest below sigma_i (an exact rescaling that keeps stored norms O(||A||) instead of growing like
//                 ||A||^i), and its per-block norm partials.
//   k_inner_qr    a cluster of CTAs: Gram-Schmidt with one reorthogonalisation pass of S A b_i against Q
//                 (Section 3, C2), the condition proxy max|r_ll|/min|r_ll| (rule C2), the running sketched residual
//                 (rule C3) and C1.  It runs on a second stream, overlapping the next step's SpMV; a step that runs
//                 past the end of the cycle is discarded.
// After the cycle: k_inner_ls solves R_k y = (Q^T S v)_k and k_inner_gemv forms z_j = B_k y_k (FP64 output).
#include "kernels.h"
#include "spmv.cuh"

#include <climits>
#include <algorithm>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace sfg {

// ---------------------------------------------------------------------------------------------------------------
// Phase 1, one thread per row: w' = A u_i fused with storing w' (global W and the shared block copy) and the
// window dot products acc_q += u_{lo+q}[r] * w'[r].  The window values and the next row group's extents are loaded
// before the row's SpMV, so they are in flight together.  Returns the thread's largest exponent of w'.
template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ int spmv_dots_scalar(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                                const MT* __restrict__ val, const VT* __restrict__ Ub, int i, int lo,
                                                int r0, int r1, AT* __restrict__ wblk, AT* __restrict__ W,
                                                AT (&acc)[NW > 0 ? NW : 1], AT& nrm) {
    const int lane = threadIdx.x & 31;
    const VT* x = Ub + (int64_t)i * n;
    int emax = 1;
    int rw = r0 + (threadIdx.x & ~31);
    int a = 0, len = 0;
    if (rw + lane < r1) {
        a = __ldg(rp + rw + lane);
        len = __ldg(rp + rw + lane + 1) - a;
    }
    for (; rw < r1; rw += blockDim.x) {  // warp-uniform loop
        const int r = rw + lane;
        const bool ok = r < r1;
        AT uw[NW > 0 ? NW : 1];
#pragma unroll
        for (int q = 0; q < NW; ++q) uw[q] = ok ? ld_plain(Ub + (int64_t)(lo + q) * n + r) : AT(0);
        AT ui;  // u_i[r] (the last window vector when there is a window) for ||u_i||^2
        if constexpr (NW > 0) ui = uw[NW - 1];
        else ui = ok ? ld_plain(x + r) : AT(0);
        const int rn = r + (int)blockDim.x;
        int an = 0, lenn = 0;
        if (rn < r1) {
            an = __ldg(rp + rn);
            lenn = __ldg(rp + rn + 1) - an;
        }
        const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
        AT sum = AT(0);
        for (int pk = 0; pk < maxlen; pk += 4) {
            switch (min(maxlen - pk, 4)) {
                case 1: row_chunk<1>(col, val, x, a, len, pk, sum); break;
                case 2: row_chunk<2>(col, val, x, a, len, pk, sum); break;
                case 3: row_chunk<3>(col, val, x, a, len, pk, sum); break;
                default: row_chunk<4>(col, val, x, a, len, pk, sum); break;
            }
        }
        if (ok) {
            W[r] = sum;
            wblk[r - r0] = sum;
        }
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += uw[q] * sum;
        nrm += ui * ui;
        emax = max(emax, exp_of(sum));
        a = an;
        len = lenn;
    }
    return emax;
}

// Phase 1 tail for the sub-warp path (w' already in shared memory): store w' and accumulate the window dots.
template <int NW, typename VT, typename AT>
__device__ __forceinline__ int dots_pass(int n, int r0, int r1, const VT* __restrict__ Ub, int lo, int i,
                                         const AT* __restrict__ wblk, AT* __restrict__ W,
                                         AT (&acc)[NW > 0 ? NW : 1], AT& nrm) {
    int emax = 1;
#pragma unroll 2
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const AT w = wblk[r - r0];
        W[r] = w;
        emax = max(emax, exp_of(w));
        const AT ui = ld_plain(Ub + (int64_t)i * n + r);
        nrm += ui * ui;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += ld_plain(Ub + (int64_t)(lo + q) * n + r) * w;
    }
    return emax;
}

// ---------------------------------------------------------------------------------------------------------------
// Shared memory: the block of w' (Bn + 1 slots of AT, slot Bn = 0 for the list padding).  FP64: the block is
// converted in place to its 64-bit fixed-point image before the sketch sums.
// At most 56 registers per thread (registers are allocated in units of 8 per thread): two 512-thread CTAs per SM
// then leave room for the sketched-QR cluster's CTAs to run beside them instead of displacing them.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(56)
    k_inner_spmv(int n, int Bn, int s, int i, int H, const int* __restrict__ rp, const int* __restrict__ col,
                 const MT* __restrict__ val, const VT* __restrict__ Ub, AT* __restrict__ W, AT* __restrict__ hpart,
                 AT* __restrict__ cpart, AT* __restrict__ normpart, const int* __restrict__ seg,
                 const uint16_t* __restrict__ ent, const CycleState* __restrict__ cyc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    __shared__ AT red[512];
    __shared__ int stop_sh, emax_sh[16];
    if (threadIdx.x == 0) stop_sh = (cyc->stopped || cyc->brk_step <= i) ? 1 : 0;
    __syncthreads();
    if (stop_sh) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    const int lo = i - NW + 1;  // window u_lo..u_i (NW = min(t, i+1))
    AT acc[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) acc[q] = AT(0);
    int emax;
    AT nrm = AT(0);  // ||u_i||^2 over the block (the vector this step multiplies)
    if constexpr (V == 1) {
        emax = spmv_dots_scalar<NW>(n, rp, col, val, Ub, i, lo, r0, r1, wblk, W, acc, nrm);
    } else {
        spmv_rows_vector<V, U, MT, VT, AT>(rp, col, val, Ub + (int64_t)i * n, r0, r1, wblk);
        __syncthreads();
        emax = dots_pass<NW>(n, r0, r1, Ub, lo, i, wblk, W, acc, nrm);
    }
    if (threadIdx.x == 0) wblk[Bn] = AT(0);
    {
        const AT v = block_sum_lean(nrm, red);
        if (threadIdx.x == 0) normpart[b] = v;
    }
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const AT v = block_sum_lean(acc[q], red);
        if (threadIdx.x == 0) hpart[(int64_t)b * kMaxTrunc + q] = v;
    }
    const int* sg = seg + (int64_t)b * s;
    if constexpr (sizeof(AT) == 8) {
        // exact fixed-point sketch sums (integer adds; the FP64 pipe stays with the SpMV)
        emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
        if (lane == 0) emax_sh[warp] = emax;
        __syncthreads();
        int Eb = 1;
        for (int q = 0; q < nw; ++q) Eb = max(Eb, emax_sh[q]);
        long long* qblk = reinterpret_cast<long long*>(wblk);
        for (int r = threadIdx.x; r <= Bn; r += blockDim.x) qblk[r] = (r < r1 - r0) ? to_fixed((double)wblk[r], Eb, H) : 0;
        __syncthreads();
        const double unit = fixed_unit(0.0, Eb, H);
        const bool bad = exp_nonfinite(0.0, Eb);
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            const long long v = sum_list(ent, sg[rr], sg[rr + 1], qblk);
            cpart[(int64_t)b * s + rr] = bad ? (AT)NAN : (AT)((double)v * unit);
        }
    } else {
        __syncthreads();
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x)
            cpart[(int64_t)b * s + rr] = sum_list(ent, sg[rr], sg[rr + 1], wblk);
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Truncated-Arnoldi update (NW = window size).  Each thread first loads its first PF rows of w' and of the window
// vectors (they do not depend on the scalars), then forms sigma_i, the coefficients and its share of the sketched
// column, so the row data are already in flight while the reductions run.
template <int NW, typename VT, typename AT>
__global__ void __launch_bounds__(512)
    k_inner_axpy(int n, int Bn, int nblk, int s, int i, int last, double sk_scale, VT* __restrict__ Ub,
                 const AT* __restrict__ W, double* __restrict__ sigma, const AT* __restrict__ normpart,
                 const AT* __restrict__ hpart, const AT* __restrict__ cpart, double* __restrict__ C,
                 double* __restrict__ hco, CycleState* __restrict__ cyc) {
    constexpr int PF = 2;
    __shared__ AT coef_sh[kMaxTrunc];
    __shared__ double sig_sh;
    __shared__ int stop_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    const int lo = i - NW + 1;
    AT wv[PF], uv[PF][NW > 0 ? NW : 1];
    if (!last) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int r = r0 + threadIdx.x + u * (int)blockDim.x;
            wv[u] = (r < r1) ? W[r] : AT(0);
#pragma unroll
            for (int q = 0; q < NW; ++q) uv[u][q] = (r < r1) ? ld_plain(Ub + (int64_t)(lo + q) * n + r) : AT(0);
        }
    }
    if (threadIdx.x == 0) stop_sh = (cyc->stopped || cyc->brk_step <= i) ? 1 : 0;
    __syncthreads();
    if (stop_sh) return;
    // sigma_i = 1/||u_i|| from the SpMV kernel's per-block partials
    if (warp == 0) {
        double sig = 1.0;
        bool bad = false;
        int why = 4;
        if (i == 0) {
            sig = sigma[0];
        } else {
            AT a = AT(0);
            for (int q = lane; q < nblk; q += 32) a += normpart[q];
            a = warp_sum(a);
            const double a2 = (double)a;
            bad = !(a2 > 0.0) || !isfinite(a2);
            why = (a2 == 0.0) ? 4 : 6;
            sig = 1.0 / sqrt(a2);
        }
        if (lane == 0) {
            sig_sh = sig;
            if (bad) {
                stop_sh = 1;
                if (b == 0) {
                    cyc->brk_reason = why;
                    atomicMin(&cyc->brk_step, i);
                }
            } else if (b == 0) {
                sigma[i] = sig;
            }
        }
    }
    __syncthreads();
    if (stop_sh) return;
    const double sig_i = sig_sh;
    // h_l = sigma_l sigma_i (u_l^T w'); the stored update uses sigma_l^2 (u_l^T w')
    if (warp < NW) {
        AT a = AT(0);
        for (int q = lane; q < nblk; q += 32) a += hpart[(int64_t)q * kMaxTrunc + warp];
        a = warp_sum(a);
        if (lane == 0) {
            const int l = lo + warp;
            const double sl = (l == i) ? sig_i : sigma[l];
            coef_sh[warp] = (AT)(sl * sl * (double)a);
            if (b == 0) hco[(int64_t)i * kMaxTrunc + warp] = sl * sig_i * (double)a;
        }
    }
    // sketched column S A b_i = sigma_i S w': one warp per sketch row across the grid
    const double csc = sk_scale * sig_i;
    for (int rr = b * nw + warp; rr < s; rr += nblk * nw) {
        AT a = AT(0);
        for (int q = lane; q < nblk; q += 32) a += cpart[(int64_t)q * s + rr];
        a = warp_sum(a);
        if (lane == 0) C[(int64_t)i * s + rr] = csc * (double)a;
    }
    if (last) return;
    __syncthreads();
    // u_{i+1} = 2^p2 (w' - sum_q coef_q u_{lo+q}), 2^p2 the power of two just below sigma_i
    int p2;
    frexp(sig_i, &p2);  // sigma_i = f * 2^p2, f in [0.5, 1)
    p2 -= 1;
    const AT sc2 = (AT)ldexp(1.0, p2);
    AT cf[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) cf[q] = coef_sh[q];
    VT* un = Ub + (int64_t)(i + 1) * n;
    auto update = [&](int r, AT u, const AT (&uq)[NW > 0 ? NW : 1]) {
#pragma unroll
        for (int q = 0; q < NW; ++q) u -= cf[q] * uq[q];
        if constexpr (sizeof(AT) == 8) u = mul_pow2((double)u, p2);
        else u = u * sc2;
        store_as(un + r, u);
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        const int r = r0 + threadIdx.x + u * (int)blockDim.x;
        if (r < r1) update(r, wv[u], uv[u]);
    }
#pragma unroll 2
    for (int r = r0 + threadIdx.x + PF * (int)blockDim.x; r < r1; r += blockDim.x) {
        AT uq[NW > 0 ? NW : 1];
#pragma unroll
        for (int q = 0; q < NW; ++q) uq[q] = ld_plain(Ub + (int64_t)(lo + q) * n + r);
        update(r, W[r], uq);
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Sketched QR update of column i on a cluster of CTAs; CTA q of the cluster owns rows [s q / nq, s (q+1) / nq) of
// Q and of the working vectors, and partial dot products are exchanged through distributed shared memory and summed
// in rank order (deterministic).  Every early exit is decided from values all CTAs of the cluster share.  CTAs are
// small (128 threads) so they fit beside the inner SpMV's CTAs, and every long FP64 dependency chain is split into
// four independent accumulators (combined in a fixed order).
__global__ void __launch_bounds__(128)
    k_inner_qr(int s, int m, int i, const double* __restrict__ C, double* __restrict__ Q, double* __restrict__ R,
               double* __restrict__ d, double* __restrict__ e, double* __restrict__ rho,
               CycleState* __restrict__ cyc) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank(), nq = (int)cl.num_blocks();
    const int rlo = (int)((int64_t)s * q / nq), rhi = (int)((int64_t)s * (q + 1) / nq), nr = rhi - rlo;
    const int nrmax = (s + nq - 1) / nq;
    extern __shared__ double qsm[];
    double* p = qsm;               // [nrmax] this CTA's rows of the working vector
    double* apart = qsm + nrmax;   // [m] partial projections over this CTA's rows
    double* a = apart + m;         // [m] full projections
    __shared__ double red[128];
    __shared__ double scal[4];
    __shared__ int code_sh;
    // state read by every CTA before the first cluster barrier (rank 0 writes it only after the last one)
    const double dmax0 = cyc->dmax, dmin0 = cyc->dmin, thr = cyc->cond_thr;
    if (q == 0 && threadIdx.x == 0) code_sh = cyc->stopped ? 1 : (cyc->brk_step <= i ? 2 : 0);
    cl.sync();
    const int code = *cl.map_shared_rank(&code_sh, 0);
    cl.sync();
    if (code) {
        if (code == 2 && q == 0 && threadIdx.x == 0) {
            cyc->stopped = 1;  // u_i has zero (or non-finite) norm: the cycle keeps k = i columns
            cyc->reason = cyc->brk_reason;
        }
        return;
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) p[r] = C[(int64_t)i * s + rlo + r];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int l = threadIdx.x; l < i; l += blockDim.x) {
            const double* ql = Q + (int64_t)l * s + rlo;
            double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
            int r = 0;
            for (; r + 4 <= nr; r += 4) {
                c0 += ql[r] * p[r];
                c1 += ql[r + 1] * p[r + 1];
                c2 += ql[r + 2] * p[r + 2];
                c3 += ql[r + 3] * p[r + 3];
            }
            for (; r < nr; ++r) c0 += ql[r] * p[r];
            apart[l] = (c0 + c1) + (c2 + c3);
        }
        cl.sync();
        for (int l = threadIdx.x; l < i; l += blockDim.x) {
            double acc = 0.0;
            for (int qq = 0; qq < nq; ++qq) acc += cl.map_shared_rank(apart, qq)[l];
            a[l] = acc;
        }
        cl.sync();  // every CTA has read the partials before the next pass overwrites them
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
            const double* qr = Q + rlo + r;
            double v0 = p[r], v1 = 0.0, v2 = 0.0, v3 = 0.0;
            int l = 0;
            for (; l + 4 <= i; l += 4) {
                v0 -= a[l] * qr[(int64_t)l * s];
                v1 -= a[l + 1] * qr[(int64_t)(l + 1) * s];
                v2 -= a[l + 2] * qr[(int64_t)(l + 2) * s];
                v3 -= a[l + 3] * qr[(int64_t)(l + 3) * s];
            }
            for (; l < i; ++l) v0 -= a[l] * qr[(int64_t)l * s];
            p[r] = (v0 + v1) + (v2 + v3);
        }
        if (q == 0)
            for (int l = threadIdx.x; l < i; l += blockDim.x)
                R[(int64_t)i * m + l] = (pass ? R[(int64_t)i * m + l] : 0.0) + a[l];
        __syncthreads();
    }
    double v2 = 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) v2 += p[r] * p[r];
    v2 = block_sum_lean(v2, red);
    if (threadIdx.x == 0) scal[0] = v2;
    cl.sync();
    double nn = 0.0;
    for (int qq = 0; qq < nq; ++qq) nn += cl.map_shared_rank(scal, qq)[0];
    const double rii = sqrt(nn);
    const double dmax = fmax(dmax0, rii);
    const double dmin = (i == 0) ? rii : fmin(dmin0, rii);
    const double kappa = (dmin > 0.0) ? dmax / dmin : INFINITY;
    if (!(kappa <= thr)) {  // C2 (also rii == 0 or NaN): drop column i, keep k = i
        if (q == 0 && threadIdx.x == 0) {
            cyc->stopped = 1;
            cyc->k = i;
            cyc->reason = (i == 0) ? 5 : 2;
        }
        cl.sync();
        return;
    }
    const double inv = 1.0 / rii;
    double dd = 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const double qv = p[r] * inv;
        p[r] = qv;
        Q[(int64_t)i * s + rlo + r] = qv;
        dd += qv * e[rlo + r];
    }
    dd = block_sum_lean(dd, red);
    if (threadIdx.x == 0) scal[1] = dd;
    cl.sync();
    double di = 0.0;
    for (int qq = 0; qq < nq; ++qq) di += cl.map_shared_rank(scal, qq)[1];
    double ee = 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const double ev = e[rlo + r] - di * p[r];
        e[rlo + r] = ev;
        ee += ev * ev;
    }
    ee = block_sum_lean(ee, red);
    if (threadIdx.x == 0) scal[2] = ee;
    cl.sync();
    double rr2 = 0.0;
    for (int qq = 0; qq < nq; ++qq) rr2 += cl.map_shared_rank(scal, qq)[2];
    const double rh = sqrt(rr2);
    if (q == 0 && threadIdx.x == 0) {
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
// y = R_k^{-1} d (back substitution, one warp), coef_l = y_l * sigma_l.
__global__ void k_inner_ls(int m, const double* __restrict__ R, const double* __restrict__ d,
                           const double* __restrict__ sigma, double* __restrict__ y, double* __restrict__ coef,
                           const CycleState* __restrict__ cyc) {
    extern __shared__ double rhs[];
    const int k = cyc->k;
    const int lane = threadIdx.x;
    for (int l = lane; l < k; l += 32) rhs[l] = d[l];
    __syncwarp();
    for (int l = k - 1; l >= 0; --l) {
        const double yl = rhs[l] / R[(int64_t)l * m + l];
        for (int q = lane; q < l; q += 32) rhs[q] -= R[(int64_t)l * m + q] * yl;
        if (lane == 0) {
            y[l] = yl;
            coef[l] = yl * sigma[l];
        }
        __syncwarp();
    }
}

// z = sum_{l<k} coef_l u_l, FP64 output.  FP64 basis: FP64 FMAs.  FP32/BF16 basis: the FP64 coefficients are
// split into two FP32 parts and the sum is carried as an unevaluated FP32 pair (TwoSum, and FMA for the exact
// product error), close to FP64 accuracy on the FP32 pipe.
template <typename VT>
__global__ void __launch_bounds__(256) k_inner_gemv(int n, const VT* __restrict__ Ub, const double* __restrict__ coef,
                                                    const CycleState* __restrict__ cyc, double* __restrict__ z) {
    __shared__ double cf[kMaxM];
    __shared__ float ch[kMaxM], clo[kMaxM];
    const int k = cyc->k;
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        const double c = coef[l];
        cf[l] = c;
        const float hi = (float)c;
        ch[l] = hi;
        clo[l] = (float)(c - (double)hi);
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(VT) == 8) {
            double acc = 0.0;
            for (int l = 0; l < k; ++l) acc += cf[l] * (double)ld_plain(Ub + (int64_t)l * n + r);
            z[r] = acc;
        } else {
            float sh = 0.f, sl = 0.f;
            for (int l = 0; l < k; ++l) {
                const float u = ld_plain(Ub + (int64_t)l * n + r);
                const float p = ch[l] * u;
                const float pe = fmaf(ch[l], u, -p) + clo[l] * u;  // exact product error + low-part term
                const float t1 = sh + p;                             // TwoSum(sh, p)
                const float bv = t1 - sh;
                const float err = (sh - (t1 - bv)) + (p - bv);
                sh = t1;
                sl += err + pe;
            }
            z[r] = (double)sh + (double)sl;
        }
    }
}

template <typename VT>
__global__ void k_export_basis(int n, int count, const VT* __restrict__ Ub, const double* __restrict__ sigma,
                               double* __restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        for (int l = 0; l < count; ++l) out[(int64_t)l * n + r] = sigma[l] * (double)ld_plain(Ub + (int64_t)l * n + r);
}

// ---------------------------------------------------------------------------------------------------------------
// Start of inner cycle j: reset the cycle state (C3 scale = FFOM residual of the previous outer step, beta at the
// first, Eq. 5), u_0 = v_j (copied into the basis storage precision), c0 = S u_0, running residual e = c0.
__global__ void k_cycle_reset(CycleState* cyc, const OuterState* ost, int j, int c3_on, double cond_thr,
                              double* sigma) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    cyc->stopped = 0;
    cyc->k = 0;
    cyc->reason = 0;
    cyc->brk_step = INT_MAX;
    cyc->brk_reason = 0;
    cyc->dmax = 0.0;
    cyc->dmin = INFINITY;
    cyc->rho = INFINITY;
    cyc->cond_thr = cond_thr;
    if (ost) {
        const double sc = (j == 0) ? ost->beta : ost->ffom;
        cyc->c3_scale = sc;
        cyc->c3_tol = ost->tol_abs;
        cyc->c3_on = (c3_on && isfinite(sc)) ? 1 : 0;
    } else {
        cyc->c3_scale = INFINITY;
        cyc->c3_tol = 0.0;
        cyc->c3_on = 0;
    }
    sigma[0] = 1.0;
}

void launch_cycle_start(const Plan& p, int j, const double* v, const double* vscale_dev, int c3_on,
                        double cond_thr) {
    k_cycle_reset<<<1, 32, 0, p.st>>>(p.cyc, j >= 0 ? p.ost : nullptr, j, c3_on, cond_thr, p.sigma);
    launch_sketch_partials(p, v, vscale_dev, p.U, p.cpart);
    launch_sketch_reduce(p, p.cpart, p.c0, p.e);
    ++g_launches;
}

template <int V, int U, int NW, typename MT, typename VT, typename AT>
static void inner_spmv_v(const Plan& p, int i, const MT* val) {
    const size_t sm = (size_t)(p.Bn + 1) * sizeof(AT);
    set_smem((const void*)k_inner_spmv<V, U, NW, MT, VT, AT>, sm);
    k_inner_spmv<V, U, NW, MT, VT, AT><<<p.nblk, 512, sm, p.st>>>(p.n, p.Bn, p.s, i, p.sk_headroom, p.rp, p.col,
                                                                 val, (const VT*)p.U, (AT*)p.W, (AT*)p.hpart,
                                                                 (AT*)p.cpart, (AT*)p.normpart, p.seg, p.ent, p.cyc);
}

template <int NW, typename MT, typename VT, typename AT>
static void inner_spmv_nw(const Plan& p, int i, const MT* val) {
    if (p.vec == 1) inner_spmv_v<1, 1, NW, MT, VT, AT>(p, i, val);
    else if (p.vec <= 8) inner_spmv_v<8, 4, NW, MT, VT, AT>(p, i, val);
    else inner_spmv_v<32, 2, NW, MT, VT, AT>(p, i, val);
}

template <typename MT, typename VT, typename AT>
static void inner_spmv_t(const Plan& p, int i, const MT* val) {
    const int nwin = (p.t > 0) ? std::min(p.t, i + 1) : 0;
    switch (nwin) {
        case 0: inner_spmv_nw<0, MT, VT, AT>(p, i, val); break;
        case 1: inner_spmv_nw<1, MT, VT, AT>(p, i, val); break;
        case 2: inner_spmv_nw<2, MT, VT, AT>(p, i, val); break;
        case 3: inner_spmv_nw<3, MT, VT, AT>(p, i, val); break;
        case 4: inner_spmv_nw<4, MT, VT, AT>(p, i, val); break;
        case 5: inner_spmv_nw<5, MT, VT, AT>(p, i, val); break;
        case 6: inner_spmv_nw<6, MT, VT, AT>(p, i, val); break;
        case 7: inner_spmv_nw<7, MT, VT, AT>(p, i, val); break;
        default: inner_spmv_nw<8, MT, VT, AT>(p, i, val); break;
    }
}

void launch_inner_spmv(const Plan& p, int i) {
    if (p.prec == kFP64) inner_spmv_t<double, double, double>(p, i, p.val);
    else if (p.prec == kFP32) inner_spmv_t<float, float, float>(p, i, p.val32);
    else inner_spmv_t<float, __nv_bfloat16, float>(p, i, p.val32);
    ++g_launches;
}

template <int NW, typename VT, typename AT>
static void inner_axpy_nw(const Plan& p, int i, bool last) {
    k_inner_axpy<NW, VT, AT><<<p.nblk, 512, 0, p.st>>>(p.n, p.Bn, p.nblk, p.s, i, last ? 1 : 0, p.sk_scale,
                                                       (VT*)p.U, (const AT*)p.W, p.sigma, (const AT*)p.normpart,
                                                       (const AT*)p.hpart, (const AT*)p.cpart, p.C, p.hco, p.cyc);
}

template <typename VT, typename AT>
static void inner_axpy_t(const Plan& p, int i, bool last) {
    const int nwin = (p.t > 0) ? std::min(p.t, i + 1) : 0;
    switch (nwin) {
        case 0: inner_axpy_nw<0, VT, AT>(p, i, last); break;
        case 1: inner_axpy_nw<1, VT, AT>(p, i, last); break;
        case 2: inner_axpy_nw<2, VT, AT>(p, i, last); break;
        case 3: inner_axpy_nw<3, VT, AT>(p, i, last); break;
        case 4: inner_axpy_nw<4, VT, AT>(p, i, last); break;
        case 5: inner_axpy_nw<5, VT, AT>(p, i, last); break;
        case 6: inner_axpy_nw<6, VT, AT>(p, i, last); break;
        case 7: inner_axpy_nw<7, VT, AT>(p, i, last); break;
        default: inner_axpy_nw<8, VT, AT>(p, i, last); break;
    }
}

void launch_inner_axpy(const Plan& p, int i, bool last) {
    if (p.prec == kFP64) inner_axpy_t<double, double>(p, i, last);
    else if (p.prec == kFP32) inner_axpy_t<float, float>(p, i, last);
    else inner_axpy_t<__nv_bfloat16, float>(p, i, last);
    ++g_launches;
}

cudaError_t launch_inner_qr(const Plan& p, int i, cudaStream_t st) {
    const int nrmax = (p.s + kQrCluster - 1) / kQrCluster;
    const size_t sm = (size_t)(nrmax + 2 * p.m) * sizeof(double);
    set_smem((const void*)k_inner_qr, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kQrCluster, 1, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kQrCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++g_launches;
    return cudaLaunchKernelEx(&cfg, k_inner_qr, p.s, p.m, i, (const double*)p.C, p.Q, p.R, p.d, p.e, p.rho, p.cyc);
}

void launch_inner_finish(const Plan& p, double* z) {
    k_inner_ls<<<1, 32, (size_t)p.m * sizeof(double), p.st>>>(p.m, p.R, p.d, p.sigma, p.y, p.coef, p.cyc);
    const int th = 256;
    const int gr = (int)std::min<int64_t>(((int64_t)p.n + th - 1) / th, 152 * 8);
    if (p.prec == kFP64) k_inner_gemv<double><<<gr, th, 0, p.st>>>(p.n, (const double*)p.U, p.coef, p.cyc, z);
    else if (p.prec == kFP32) k_inner_gemv<float><<<gr, th, 0, p.st>>>(p.n, (const float*)p.U, p.coef, p.cyc, z);
    else k_inner_gemv<__nv_bfloat16><<<gr, th, 0, p.st>>>(p.n, (const __nv_bfloat16*)p.U, p.coef, p.cyc, z);
    g_launches += 2;
}

void launch_export_basis(const Plan& p, double* out, int count) {
    const int th = 256;
    const int gr = (int)std::min<int64_t>(((int64_t)p.n + th - 1) / th, 152 * 8);
    if (p.prec == kFP64) k_export_basis<double><<<gr, th, 0, p.st>>>(p.n, count, (const double*)p.U, p.sigma, out);
    else if (p.prec == kFP32) k_export_basis<float><<<gr, th, 0, p.st>>>(p.n, count, (const float*)p.U, p.sigma, out);
    else k_export_basis<__nv_bfloat16><<<gr, th, 0, p.st>>>(p.n, count, (const __nv_bfloat16*)p.U, p.sigma, out);
    ++g_launches;
}

}  // namespace sfg
