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
#include "kernels.h"
#include "spmv.cuh"

#include <climits>
#include <algorithm>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace sfg {

// Template value of k_inner_spmv's lanes-per-row parameter for one thread per row reading the SELL-32 copy of A
// (the FP64 inner cycle); 1 is one thread per row reading the CSR arrays.
constexpr int kVecSell = -1;

__device__ __forceinline__ bool cycle_idle(const Plan& P, int p, int i) {
    const CycleState* c = P.cyc + p;
    return c->stopped || c->brk_step <= i || (P.pflag[p] & 1);
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// ---------------------------------------------------------------------------------------------------------------
// Entries pk .. pk+CNT-1 of the thread's row in the SELL-32 copy (cp, vp: the lane's first entry; consecutive
// entries 32 apart, so each load is coalesced across the warp); entries past the row's end (rl) are not gathered.
template <int CNT, typename MT, typename XT, typename AT>
__device__ __forceinline__ void sell_chunk(const int* __restrict__ cp, const MT* __restrict__ vp,
                                           const XT* __restrict__ x, int rl, int pk, AT& sum) {
    int c[CNT];
    AT v[CNT];
#pragma unroll
    for (int q = 0; q < CNT; ++q) {
        c[q] = __ldg(cp + (pk + q) * 32);
        v[q] = (AT)__ldg(vp + (pk + q) * 32);
    }
#pragma unroll
    for (int q = 0; q < CNT; ++q)
        if (pk + q < rl) sum += v[q] * load_as(x + c[q], AT());
}

// Phase 1, one thread per row, from the SELL-32 copy of A: w' = A u_i over the block (vector rows v0 .. v0+len,
// whose matrix rows start the list block's first slice sb; warp rows kw .. kw+31 are slice sb + kw/32), fused with
// storing w' (global W and the shared block copy), the window dot products acc_q += u_{lo+q}[r] * w'[r] and
// ||u_i||^2.  Each row is summed in entry order, the warp issuing as many FMAs as its slice is wide.  The window
// values and the next slice's extent are loaded before the row's SpMV, so they are in flight together.  Returns
// the thread's largest exponent of w'.
template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ int spmv_dots_sell(int N, const int* __restrict__ soff, const uint8_t* __restrict__ slen,
                                              const int* __restrict__ scol, const MT* __restrict__ sval, int sb,
                                              const VT* __restrict__ Ub, int i, int lo, int v0, int len, int cs,
                                              AT* __restrict__ wblk, AT* __restrict__ W, AT (&acc)[NW > 0 ? NW : 1],
                                              AT& nrm) {
    const int lane = threadIdx.x & 31;
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    const VT* x = Ub + (int64_t)i * N;
    const VT* xs = x + cs;  // gather base: vector index of matrix column c is c + cs
    int emax = 1;
    int kw = threadIdx.x & ~31;
    int o0 = 0, o1 = 0, rl = 0;
    if (kw < len) {
        const int sid = sb + (kw >> 5);
        o0 = __ldg(soff + sid);
        o1 = __ldg(soff + sid + 1);
        rl = __ldg(slen + (int64_t)sid * 32 + lane);
    }
    for (; kw < len; kw += blockDim.x) {  // warp-uniform loop over the block's slices
        const int k = kw + lane;
        const bool ok = k < len;
        const int r = v0 + k;
        AT uw[NW > 0 ? NW : 1];
#pragma unroll
        for (int q = 0; q < NW; ++q) uw[q] = ok ? ld_keep(Ub + (int64_t)(lo + q) * N + r, pol) : AT(0);
        AT ui;  // u_i[r] (the last window vector when there is a window) for ||u_i||^2
        if constexpr (NW > 0) ui = uw[NW - 1];
        else ui = ok ? ld_plain(x + r) : AT(0);
        const int kn = kw + (int)blockDim.x;
        int o0n = 0, o1n = 0, rln = 0;
        if (kn < len) {
            const int sid = sb + (kn >> 5);
            o0n = __ldg(soff + sid);
            o1n = __ldg(soff + sid + 1);
            rln = __ldg(slen + (int64_t)sid * 32 + lane);
        }
        const int w = o1 - o0;
        // every 128-byte line of the slice's columns and values requested at once (one line per lane; w <= 16
        // entries, so at most 32 lines of FP64 values): the later chunks' loads then find their lines in flight
        // instead of starting another round trip to memory each
        if (lane < w) prefetch_l1(scol + (int64_t)(o0 + lane) * 32);
        if (lane < w * (int)(sizeof(MT) / 4)) prefetch_l1(reinterpret_cast<const char*>(sval + (int64_t)o0 * 32) + lane * 128);
        const int* cp = scol + (int64_t)o0 * 32 + lane;
        const MT* vp = sval + (int64_t)o0 * 32 + lane;
        AT sum = AT(0);
        for (int pk = 0; pk < w; pk += 4) {
            switch (min(w - pk, 4)) {
                case 1: sell_chunk<1>(cp, vp, xs, rl, pk, sum); break;
                case 2: sell_chunk<2>(cp, vp, xs, rl, pk, sum); break;
                case 3: sell_chunk<3>(cp, vp, xs, rl, pk, sum); break;
                default: sell_chunk<4>(cp, vp, xs, rl, pk, sum); break;
            }
        }
        if (ok) {
            st_keep(W + r, sum, pol);
            wblk[k] = sum;
        }
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += uw[q] * sum;
        nrm += ui * ui;
        emax = max(emax, exp_of(sum));
        o0 = o0n;
        o1 = o1n;
        rl = rln;
    }
    return emax;
}

// ---------------------------------------------------------------------------------------------------------------
// Phase 1, one thread per row: w' = A u_i over the block (vector rows v0 .. v0+len = matrix rows v0-cs ..) fused
// with storing w' (global W and the shared block copy), the window dot products acc_q += u_{lo+q}[r] * w'[r] and
// ||u_i||^2.  The window values and the next row group's extents are loaded before the row's SpMV, so they are in
// flight together.  Returns the thread's largest exponent of w'.
template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ int spmv_dots_scalar(int N, const int* __restrict__ rp, const int* __restrict__ col,
                                                const MT* __restrict__ val, const VT* __restrict__ Ub, int i, int lo,
                                                int v0, int len, int cs, AT* __restrict__ wblk, AT* __restrict__ W,
                                                AT (&acc)[NW > 0 ? NW : 1], AT& nrm) {
    const int lane = threadIdx.x & 31;
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    const VT* x = Ub + (int64_t)i * N;
    const VT* xs = x + cs;                // gather base: vector index of matrix column c is c + cs
    const int* rpm = rp + (v0 - cs);      // row pointers of the block's matrix rows
    int emax = 1;
    int kw = threadIdx.x & ~31;
    int a = 0, rl = 0;
    if (kw + lane < len) {
        a = __ldg(rpm + kw + lane);
        rl = __ldg(rpm + kw + lane + 1) - a;
    }
    for (; kw < len; kw += blockDim.x) {  // warp-uniform loop over the block's rows
        const int k = kw + lane;
        const bool ok = k < len;
        const int r = v0 + k;
        AT uw[NW > 0 ? NW : 1];
#pragma unroll
        for (int q = 0; q < NW; ++q) uw[q] = ok ? ld_keep(Ub + (int64_t)(lo + q) * N + r, pol) : AT(0);
        AT ui;  // u_i[r] (the last window vector when there is a window) for ||u_i||^2
        if constexpr (NW > 0) ui = uw[NW - 1];
        else ui = ok ? ld_plain(x + r) : AT(0);
        const int kn = k + (int)blockDim.x;
        int an = 0, rln = 0;
        if (kn < len) {
            an = __ldg(rpm + kn);
            rln = __ldg(rpm + kn + 1) - an;
        }
        const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)rl);
        AT sum = AT(0);
        for (int pk = 0; pk < maxlen; pk += 4) {
            switch (min(maxlen - pk, 4)) {
                case 1: row_chunk<1>(col, val, xs, a, rl, pk, sum); break;
                case 2: row_chunk<2>(col, val, xs, a, rl, pk, sum); break;
                case 3: row_chunk<3>(col, val, xs, a, rl, pk, sum); break;
                default: row_chunk<4>(col, val, xs, a, rl, pk, sum); break;
            }
        }
        if (ok) {
            st_keep(W + r, sum, pol);
            wblk[k] = sum;
        }
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += uw[q] * sum;
        nrm += ui * ui;
        emax = max(emax, exp_of(sum));
        a = an;
        rl = rln;
    }
    return emax;
}

// Phase 1 tail for the sub-warp path (w' already in shared memory): store w', accumulate the window dots and
// ||u_i||^2.
template <int NW, typename VT, typename AT>
__device__ __forceinline__ int dots_pass(int N, int v0, int len, const VT* __restrict__ Ub, int lo, int i,
                                         const AT* __restrict__ wblk, AT* __restrict__ W,
                                         AT (&acc)[NW > 0 ? NW : 1], AT& nrm) {
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    int emax = 1;
#pragma unroll 2
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const int r = v0 + k;
        const AT w = wblk[k];
        st_keep(W + r, w, pol);
        emax = max(emax, exp_of(w));
        const AT ui = ld_keep(Ub + (int64_t)i * N + r, pol);
        nrm += ui * ui;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += ld_keep(Ub + (int64_t)(lo + q) * N + r, pol) * w;
    }
    return emax;
}

// ---------------------------------------------------------------------------------------------------------------
// Shared memory: the block of w' (Bn + 1 slots of AT, slot Bn = 0 for the list padding).  FP64: the block is
// converted in place to its 64-bit fixed-point image before the sketch sums.
// At most 56 registers per thread (registers are allocated in units of 8 per thread): two 512-thread CTAs per SM
// then leave room for the sketched-QR cluster's CTAs to run beside them instead of displacing them.
// Returns false (every thread of the CTA alike) when the block's problem has no step i to take.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ bool inner_spmv_block(const Plan& P, int i, const MT* __restrict__ val,
                                                 AT* __restrict__ wblk) {
    __shared__ AT red[512];
    __shared__ int stop_sh, emax_sh[16];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    if (threadIdx.x == 0) stop_sh = cycle_idle(P, bi.prob, i) ? 1 : 0;
    __syncthreads();
    if (stop_sh) return false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s = P.s, Bn = P.Bn, N = P.N;
    const VT* Ub = (const VT*)P.U;
    AT* W = (AT*)P.W;
    const int lo = i - NW + 1;  // window u_lo..u_i (NW = min(t, i+1))
    AT acc[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) acc[q] = AT(0);
    int emax;
    AT nrm = AT(0);  // ||u_i||^2 over the block (the vector this step multiplies)
    if constexpr (V == kVecSell) {
        emax = spmv_dots_sell<NW>(N, P.sl_off, P.sl_len, P.sl_col, val, P.sl_base[bi.list], Ub, i, lo, bi.v0,
                                  bi.len, bi.cs, wblk, W, acc, nrm);
    } else if constexpr (V == 1) {
        emax = spmv_dots_scalar<NW>(N, P.rp, P.col, val, Ub, i, lo, bi.v0, bi.len, bi.cs, wblk, W, acc, nrm);
    } else {
        const int m0 = bi.v0 - bi.cs;
        int n0, n01;
        block_bins(P, bi, n0, n01);
        spmv_rows_to_smem<V, U, MT, VT, AT>(P.rp, P.col, val, Ub + (int64_t)i * N + bi.cs, m0, m0 + bi.len, wblk,
                                            P.perm, n0, n01);
        __syncthreads();
        emax = dots_pass<NW>(N, bi.v0, bi.len, Ub, lo, i, wblk, W, acc, nrm);
    }
    if (threadIdx.x == 0) wblk[Bn] = AT(0);
    // block sums of ||u_i||^2 and the window dots in one round: each warp's sums (shuffle trees), then the warps'
    // partials in warp order; the block's largest exponent of w' with them
    {
        AT (*red2)[16] = reinterpret_cast<AT (*)[16]>(red);  // [NW + 1][16]
        const AT v = warp_sum(nrm);
        if (lane == 0) red2[0][warp] = v;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const AT d = warp_sum(acc[q]);
            if (lane == 0) red2[1 + q][warp] = d;
        }
        emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
        if (lane == 0) emax_sh[warp] = emax;
        __syncthreads();
        if (threadIdx.x <= NW) {
            AT t = AT(0);
            for (int w = 0; w < nw; ++w) t += red2[threadIdx.x][w];
            if (threadIdx.x == 0) ((AT*)P.normpart)[b] = t;
            else ((AT*)P.hpart)[(int64_t)b * kMaxTrunc + threadIdx.x - 1] = t;
        }
    }
    const int* sg = P.seg + (int64_t)bi.list * s;
    AT* cpart = (AT*)P.cpart;
    if constexpr (sizeof(AT) == 8) {
        // exact fixed-point sketch sums (integer adds; the FP64 pipe stays with the SpMV)
        int Eb = 1;
        for (int q = 0; q < nw; ++q) Eb = max(Eb, emax_sh[q]);
        const int H = P.sk_headroom;
        long long* qblk = reinterpret_cast<long long*>(wblk);
        for (int r = threadIdx.x; r <= Bn; r += blockDim.x)
            qblk[r] = (r < bi.len) ? to_fixed((double)wblk[r], Eb, H) : 0;
        __syncthreads();
        const double unit = fixed_unit(0.0, Eb, H);
        const bool bad = exp_nonfinite(0.0, Eb);
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            const long long v = sum_list(P.ent, sg[rr], sg[rr + 1], qblk);
            cpart[(int64_t)b * s + rr] = bad ? (AT)NAN : (AT)((double)v * unit);
        }
    } else {
        __syncthreads();
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x)
            cpart[(int64_t)b * s + rr] = sum_list(P.ent, sg[rr], sg[rr + 1], wblk);
    }
    return true;
}

template <int V, int U, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(56) k_inner_spmv(const Plan P, int i, const MT* __restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    inner_spmv_block<V, U, NW, MT, VT, AT>(P, i, val, reinterpret_cast<AT*>(smem_raw));
}

// ---------------------------------------------------------------------------------------------------------------
// Grouped form of k_inner_spmv for matrices with short rows (one thread per row): one CTA serves the same row block
// of up to G problems that are right-hand sides of one system (the group's member blocks), so the CSR entries, the
// row pointers and the sketch gather lists are read once for all members.  Each member gets what k_inner_spmv
// computes for its block: w' stored, window dots and ||u_i||^2 partials (block sums formed warp by warp), and the
// per-block sketch partials.  Members whose cycle has stopped are skipped.
template <int CNT, int G, typename MT, typename XT, typename AT>
__device__ __forceinline__ void row_chunk_g(const int* __restrict__ col, const MT* __restrict__ val,
                                            const XT* __restrict__ x, int dn, unsigned act, int a, int len, int pk,
                                            AT (&sum)[G]) {
    int c[CNT];
    AT v[CNT];
#pragma unroll
    for (int q = 0; q < CNT; ++q) {
        if (pk + q < len) {
            c[q] = __ldg(col + a + pk + q);
            v[q] = (AT)__ldg(val + a + pk + q);
        }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) {
        if (act & (1u << j)) {
#pragma unroll
            for (int q = 0; q < CNT; ++q)
                if (pk + q < len) sum[j] += v[q] * load_as(x + j * dn + c[q], AT());
        }
    }
}

template <int G, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(sizeof(AT) == 8 ? 64 : 56) k_inner_spmv_grp(const Plan P, int i, const MT* __restrict__ val) {
    constexpr int NV = NW + 1;  // reduced values per member: ||u_i||^2 and the window dots
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ AT red[G * NV][16];
    __shared__ int emax_sh[G][16];
    __shared__ int mb_sh[G], mv0_sh[G], mcs_sh[G];
    __shared__ unsigned act_sh;
    const int gi = blockIdx.x;
    const int gb = P.grp_b[gi], gn = P.grp_n[gi], gst = P.grp_st[gi];
    if (threadIdx.x < G) {
        const int j = threadIdx.x;
        const int b = gb + min(j, gn - 1) * gst;
        mb_sh[j] = b;
        mv0_sh[j] = P.blk_v0[b];
        mcs_sh[j] = P.blk_cs[b];
    }
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int j = 0; j < gn; ++j)
            if (!cycle_idle(P, P.blk_prob[gb + j * gst], i)) a |= 1u << j;
        act_sh = a;
    }
    __syncthreads();
    const unsigned act = act_sh;
    if (!act) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s = P.s, Bn = P.Bn, N = P.N, SB = Bn + 1;
    const int len = P.blk_len[gb], list = P.blk_list[gb];
    const int m0 = mv0_sh[0] - mcs_sh[0];
    const VT* Ub = (const VT*)P.U;
    AT* W = (AT*)P.W;
    AT* wb = reinterpret_cast<AT*>(smem_raw);  // member j: wb[j * SB .. j * SB + Bn]
    const int lo = i - NW + 1;
    // members are consecutive right-hand sides of one system: their vector rows are dn apart
    const int dn = (gn > 1) ? mv0_sh[1] - mv0_sh[0] : 0;
    const int v00 = mv0_sh[0];
    const VT* xs = Ub + (int64_t)i * N + mcs_sh[0];
    AT acc[G][NW > 0 ? NW : 1], nrm[G];
    int emax[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        nrm[j] = AT(0);
        emax[j] = 1;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[j][q] = AT(0);
    }
    const int* rpm = P.rp + m0;
    int kw = threadIdx.x & ~31;
    int a = 0, rl = 0;
    if (kw + lane < len) {
        a = __ldg(rpm + kw + lane);
        rl = __ldg(rpm + kw + lane + 1) - a;
    }
    for (; kw < len; kw += blockDim.x) {  // warp-uniform loop over the block's rows
        const int k = kw + lane;
        const bool ok = k < len;
        const int kn = k + (int)blockDim.x;
        int an = 0, rln = 0;
        if (kn < len) {
            an = __ldg(rpm + kn);
            rln = __ldg(rpm + kn + 1) - an;
        }
        const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)rl);
        AT sum[G];
#pragma unroll
        for (int j = 0; j < G; ++j) sum[j] = AT(0);
        for (int pk = 0; pk < maxlen; pk += 4) {
            switch (min(maxlen - pk, 4)) {
                case 1: row_chunk_g<1, G>(P.col, val, xs, dn, act, a, rl, pk, sum); break;
                case 2: row_chunk_g<2, G>(P.col, val, xs, dn, act, a, rl, pk, sum); break;
                case 3: row_chunk_g<3, G>(P.col, val, xs, dn, act, a, rl, pk, sum); break;
                default: row_chunk_g<4, G>(P.col, val, xs, dn, act, a, rl, pk, sum); break;
            }
        }
        // window values after the SpMV (fewer live registers than prefetching them for every member)
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (act & (1u << j)) {
                const int r = v00 + j * dn + k;
                if (ok) {
                    W[r] = sum[j];
                    wb[j * SB + k] = sum[j];
                }
                AT ui = AT(0);
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    const AT u = ok ? ld_plain(Ub + (int64_t)(lo + q) * N + r) : AT(0);
                    acc[j][q] += u * sum[j];
                    ui = u;
                }
                if constexpr (NW == 0) ui = ok ? ld_plain(Ub + (int64_t)i * N + r) : AT(0);
                nrm[j] += ui * ui;
                emax[j] = max(emax[j], exp_of(sum[j]));
            }
        }
        a = an;
        rl = rln;
    }
    // block sums (warp by warp, then the warps' partials in order) of ||u_i||^2 and the window dots
#pragma unroll
    for (int j = 0; j < G; ++j) {
        if (act & (1u << j)) {
            const AT v = warp_sum(nrm[j]);
            if (lane == 0) red[j * NV][warp] = v;
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                const AT d = warp_sum(acc[j][q]);
                if (lane == 0) red[j * NV + 1 + q][warp] = d;
            }
            if constexpr (sizeof(AT) == 8) {
                const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax[j]);
                if (lane == 0) emax_sh[j][warp] = e;
            }
            if (threadIdx.x == 0) wb[j * SB + Bn] = AT(0);
        }
    }
    __syncthreads();
    if (threadIdx.x < G * NV) {
        const int j = threadIdx.x / NV, v = threadIdx.x % NV;
        if (act & (1u << j)) {
            AT t = AT(0);
            for (int w = 0; w < nw; ++w) t += red[threadIdx.x][w];
            const int b = mb_sh[j];
            if (v == 0) ((AT*)P.normpart)[b] = t;
            else ((AT*)P.hpart)[(int64_t)b * kMaxTrunc + v - 1] = t;
        }
    }
    const int* sg = P.seg + (int64_t)list * s;
    AT* cpart = (AT*)P.cpart;
    if constexpr (sizeof(AT) == 8) {
        // exact fixed-point sketch sums per member (relative to the member's block maximum)
        long long* qb = reinterpret_cast<long long*>(wb);
        const int H = P.sk_headroom;
        int Eb[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            Eb[j] = 1;
            if (act & (1u << j))
                for (int q = 0; q < nw; ++q) Eb[j] = max(Eb[j], emax_sh[j][q]);
        }
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (act & (1u << j))
                for (int r = threadIdx.x; r <= Bn; r += blockDim.x)
                    qb[j * SB + r] = (r < len) ? to_fixed((double)wb[j * SB + r], Eb[j], H) : 0;
        __syncthreads();
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            long long sums[G];
            sum_list_g<G>(P.ent, sg[rr], sg[rr + 1], qb, SB, act, sums);
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (act & (1u << j))
                    cpart[(int64_t)mb_sh[j] * s + rr] =
                        exp_nonfinite(0.0, Eb[j]) ? (AT)NAN : (AT)((double)sums[j] * fixed_unit(0.0, Eb[j], H));
        }
    } else {
        __syncthreads();
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            AT sums[G];
            sum_list_g<G>(P.ent, sg[rr], sg[rr + 1], wb, SB, act, sums);
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (act & (1u << j)) cpart[(int64_t)mb_sh[j] * s + rr] = sums[j];
        }
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Waits until the grid counter reaches target (acquire), polling with a growing sleep; after kGridWaitPolls polls it
// gives up and sets *fail.  Once a wait of the cycle has given up, later ones return at once.
constexpr int kGridWaitPolls = 1 << 20;  // about a second of polls (256 ns sleeps plus an L2 round trip each)
__device__ __forceinline__ void grid_wait(unsigned long long* ctr, unsigned long long target, unsigned long long* fail) {
    unsigned long long f;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(f) : "l"(fail) : "memory");
    if (f) return;
    unsigned ns = 32;
    for (int it = 0; it < kGridWaitPolls; ++it) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) return;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    atomicOr(fail, 1ull);
}

// ---------------------------------------------------------------------------------------------------------------
// Lane-strided sum of the per-block partials x[q * stride] for blocks q in [b0, b1) (lane l takes q = b0 + l,
// b0 + l + 32, ... in increasing order, then a shuffle tree), with every load of a lane issued before the first add.
// The loads bypass L1: in the fused step the partials come from other CTAs of the same launch.
template <typename AT>
__device__ __forceinline__ AT block_partials_sum(const AT* __restrict__ x, int64_t stride, int b0, int b1, int lane) {
    constexpr int U = 4;
    AT a = AT(0);
    for (int q0 = b0 + lane; q0 < b1; q0 += 32 * U) {
        AT t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) t[u] = (q0 + 32 * u < b1) ? __ldcg(x + (int64_t)(q0 + 32 * u) * stride) : AT(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (q0 + 32 * u < b1) a += t[u];
    }
    return warp_sum(a);
}

// Truncated-Arnoldi update (NW = window size).  Each thread first loads its first PF rows of w' and of the window
// vectors (they do not depend on the scalars); meanwhile warp 0 sums the problem's ||u_i||^2 partials and warps
// 1..NW its window-dot partials, each with all loads in flight at once.  After one barrier thread 0 forms sigma_i
// and the coefficients; after a second, the sketched column S A b_i (one warp per sketch row, rows spread over all
// of the problem's blocks) and the row update.
// Three 512-thread CTAs per SM (at most 42 registers; batches run many waves of blocks) for windows up to 3, two
// for wider windows, which would spill within 42.
// wsm: the block of w' in shared memory (the fused step, FP32/BF16), else null (w' read from W).  FUSED: the block's
// partials of this step come from other CTAs of the same launch; thread 0 waits for all of them (target arrivals
// at the step's grid counter) after the prefetch.
template <int NW, typename VT, typename AT, bool FUSED>
__device__ __forceinline__ void inner_axpy_block(const Plan& P, int i, int last, const AT* __restrict__ wsm,
                                                 unsigned long long target) {
    // rows per thread loaded before the scalars (PF) and per round of the row loop (UR; all loads of a round are
    // issued before its stores): the fused step has the whole 56-register budget here, the update kernel 42
    constexpr bool WIDE = (sizeof(AT) == 8 && NW >= 3);
    constexpr int PF = FUSED ? (WIDE ? 2 : 4) : ((sizeof(AT) == 8 && NW >= 5) ? 1 : 2);
    constexpr int UR = FUSED ? (WIDE ? 2 : 4) : ((sizeof(AT) == 8 && NW >= 4) ? 1 : 2);
    __shared__ AT coef_sh[kMaxTrunc];
    __shared__ AT part_sh[kMaxTrunc + 1];
    __shared__ double sig_sh;
    __shared__ int stop_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    const int p = bi.prob;
    const int N = P.N, s = P.s, m = P.m;
    VT* Ub = (VT*)P.U;
    const AT* W = (const AT*)P.W;
    const int lo = i - NW + 1;
    AT wv[PF], uv[PF][NW > 0 ? NW : 1];
    if (!last) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int k = threadIdx.x + u * (int)blockDim.x;
            const int r = bi.v0 + k;
            wv[u] = (k < bi.len) ? (wsm ? wsm[k] : W[r]) : AT(0);
#pragma unroll
            for (int q = 0; q < NW; ++q)
                uv[u][q] = (k < bi.len) ? ld_plain(Ub + (int64_t)(lo + q) * N + r) : AT(0);
        }
    }
    if constexpr (FUSED) {
        if (threadIdx.x == 0) grid_wait(P.gsync, target, P.gsync + 1);
        __syncthreads();
    }
    if (threadIdx.x == 0) stop_sh = cycle_idle(P, p, i) ? 1 : 0;
    const int b0 = P.prob_b0[p], b1 = P.prob_b0[p + 1];
    // ||u_i||^2 (warp 0; sigma_0 is known at i = 0) and the window dots u_l^T w' (warp 1 + q) over the blocks
    if (warp == 0 && i > 0) {
        const AT a = block_partials_sum((const AT*)P.normpart, 1, b0, b1, lane);
        if (lane == 0) part_sh[0] = a;
    } else if (warp >= 1 && warp <= NW) {
        const AT a = block_partials_sum((const AT*)P.hpart + (warp - 1), kMaxTrunc, b0, b1, lane);
        if (lane == 0) part_sh[warp] = a;
    }
    __syncthreads();
    if (stop_sh) return;
    const bool lead = (b == b0);  // the problem's first block writes its scalars
    double* sigma = P.sigma + (int64_t)p * (m + 1);
    if (threadIdx.x == 0) {
        // sigma_i = 1/||u_i||
        double sig = 1.0;
        bool bad = false;
        int why = 4;
        if (i == 0) {
            sig = sigma[0];
        } else {
            const double a2 = (double)part_sh[0];
            bad = !(a2 > 0.0) || !isfinite(a2);
            why = (a2 == 0.0) ? 4 : 6;
            sig = 1.0 / sqrt(a2);
        }
        sig_sh = sig;
        if (bad) {
            stop_sh = 1;
            if (lead) {
                CycleState* cyc = P.cyc + p;
                cyc->brk_reason = why;
                atomicMin(&cyc->brk_step, i);
            }
        } else {
            if (lead) sigma[i] = sig;
            // h_l = sigma_l sigma_i (u_l^T w'); the stored update uses sigma_l^2 (u_l^T w')
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                const int l = lo + q;
                const double a = (double)part_sh[1 + q];
                const double sl = (l == i) ? sig : sigma[l];
                coef_sh[q] = (AT)(sl * sl * a);
                if (lead) P.hco[((int64_t)p * m + i) * kMaxTrunc + q] = sl * sig * a;
            }
        }
    }
    __syncthreads();
    if (stop_sh) return;
    const double sig_i = sig_sh;
    // sketched column S A b_i = sigma_i S w': sketch row rr to warp rr / nb of the problem's block rr % nb
    const double csc = P.sk_scale * sig_i;
    const int nb = b1 - b0;
    for (int rr = warp * nb + (b - b0); rr < s; rr += nw * nb) {
        const AT a = block_partials_sum((const AT*)P.cpart + rr, s, b0, b1, lane);
        if (lane == 0) P.C[((int64_t)p * m + i) * s + rr] = csc * (double)a;
    }
    if (last) return;
    // u_{i+1} = 2^p2 (w' - sum_q coef_q u_{lo+q}), 2^p2 the power of two just below sigma_i
    int p2;
    frexp(sig_i, &p2);  // sigma_i = f * 2^p2, f in [0.5, 1)
    p2 -= 1;
    const AT sc2 = (AT)ldexp(1.0, p2);
    AT cf[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) cf[q] = coef_sh[q];
    VT* un = Ub + (int64_t)(i + 1) * N;
    const unsigned long long pol = l2_keep_policy();
    auto update = [&](int r, AT u, const AT (&uq)[NW > 0 ? NW : 1]) {
#pragma unroll
        for (int q = 0; q < NW; ++q) u -= cf[q] * uq[q];
        if constexpr (sizeof(AT) == 8) u = mul_pow2((double)u, p2);
        else u = u * sc2;
        st_keep(un + r, u, pol);  // the next step gathers it and reads it as a window row
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        const int k = threadIdx.x + u * (int)blockDim.x;
        if (k < bi.len) update(bi.v0 + k, wv[u], uv[u]);
    }
    for (int k0 = threadIdx.x + PF * (int)blockDim.x; k0 < bi.len; k0 += UR * (int)blockDim.x) {
        AT wr[UR], uq[UR][NW > 0 ? NW : 1];
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int k = k0 + u * (int)blockDim.x;
            const bool ok = k < bi.len;
            const int r = bi.v0 + k;
            wr[u] = ok ? (wsm ? wsm[k] : W[r]) : AT(0);
#pragma unroll
            for (int q = 0; q < NW; ++q) uq[u][q] = ok ? ld_plain(Ub + (int64_t)(lo + q) * N + r) : AT(0);
        }
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int k = k0 + u * (int)blockDim.x;
            if (k < bi.len) update(bi.v0 + k, wr[u], uq[u]);
        }
    }
}

template <int NW, typename VT, typename AT>
__global__ void __launch_bounds__(512, (NW <= 3) ? 3 : 2) k_inner_axpy(const Plan P, int i, int last) {
    inner_axpy_block<NW, VT, AT, false>(P, i, last, nullptr, 0);
}

// ---------------------------------------------------------------------------------------------------------------
// One inner step in one launch, for plans whose row blocks all fit on the GPU at once (one wave): the fused SpMV +
// dots + sketch partials, then a grid-wide arrival (every CTA, also one with no step to take), then, once all of the
// launch's partials are written, the truncated-Arnoldi update of the CTA's own rows.  Every CTA of the launch is
// resident at the same time (the host launches it only when the occupancy allows all blocks at once, beside the
// sketched-QR cluster), so the wait ends; it gives up after a bounded number of polls and raises the plan's sync
// flag, which the outer step turns into an error.  The arithmetic and its order are those of the two kernels.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(56) k_inner_step(const Plan P, int i, const MT* __restrict__ val, int last) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    __shared__ unsigned long long target_sh;
    const bool active = inner_spmv_block<V, U, NW, MT, VT, AT>(P, i, val, wblk);
    __threadfence();  // this thread's partials are visible device-wide before the CTA arrives
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long old = atomicAdd(P.gsync, 1ull);
        target_sh = (old / gridDim.x + 1) * (unsigned long long)gridDim.x + (unsigned long long)P.gwait_extra;
    }
    if (!active) return;
    // FP64: the shared block now holds the fixed-point image of w', so w' is read back from W
    inner_axpy_block<NW, VT, AT, true>(P, i, last, sizeof(AT) == 8 ? nullptr : wblk, target_sh);
}

// ---------------------------------------------------------------------------------------------------------------
// Sketched QR update of column i, one cluster of nq CTAs per problem (cluster index = problem); CTA q owns rows
// [s q / nq, s (q+1) / nq) of Q and of the working vectors.  Partial dot products go through distributed shared
// memory and are summed in rank order (deterministic, the same values in every CTA, so every decision is taken
// identically everywhere).  Five cluster barriers per update: one per Gram-Schmidt pass (the two passes' partials
// live in separate buffers), one for ||p||^2 and p^T e together (d_i = p^T e / r_ii), one for the updated residual
// norm, and a last one before any CTA leaves.  Each CTA reads the stop state itself (written by earlier launches;
// the one field another stream may change meanwhile, the breakdown step, only ever moves to values above i).
// CTAs are small (128 threads) so they fit beside the inner SpMV's CTAs, and every long FP64 dependency chain is
// split into four independent accumulators (combined in a fixed order).
__device__ __forceinline__ double qr_rank_sum(cg::cluster_group& cl, double* base, int off, int nq) {
    double v[kQrCluster];
#pragma unroll
    for (int r2 = 0; r2 < kQrCluster; ++r2) v[r2] = (r2 < nq) ? cl.map_shared_rank(base, r2)[off] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int r2 = 0; r2 < kQrCluster; ++r2) acc += v[r2];
    return acc;
}

// Sum over the CTA's 128 threads of v (warp trees, then the 4 warps in order); valid in every thread.
__device__ __forceinline__ double qr_block_sum(double v, double* red4) {
    v = warp_sum(v);
    __syncthreads();  // red4 is free (its previous values have been read)
    if ((threadIdx.x & 31) == 0) red4[threadIdx.x >> 5] = v;
    __syncthreads();
    return (red4[0] + red4[1]) + (red4[2] + red4[3]);
}

__global__ void __launch_bounds__(128) k_inner_qr(const Plan P, int i) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank(), nq = (int)cl.num_blocks();
    const int prob = blockIdx.x / nq;
    const int s = P.s, m = P.m;
    const double* __restrict__ C = P.C + (int64_t)prob * m * s;
    double* __restrict__ Q = P.Q + (int64_t)prob * m * s;
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
    // the cycle state as earlier launches left it (the same for every CTA of the cluster)
    const double dmax0 = cyc->dmax, dmin0 = cyc->dmin, thr = cyc->cond_thr;
    const int code = (cyc->stopped || (P.pflag[prob] & 1)) ? 1 : (cyc->brk_step <= i ? 2 : 0);
    if (code) {
        if (code == 2 && q == 0 && threadIdx.x == 0) {
            cyc->stopped = 1;  // u_i has zero (or non-finite) norm: the cycle keeps k = i columns
            cyc->reason = cyc->brk_reason;
        }
        return;  // the whole cluster returns
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) p[r] = C[(int64_t)i * s + rlo + r];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        double* ap = apart + pass * m;
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
            ap[l] = (c0 + c1) + (c2 + c3);
        }
        cl.sync();  // this pass's partials of every CTA are in place
        for (int l = threadIdx.x; l < i; l += blockDim.x) a[l] = qr_rank_sum(cl, ap, l, nq);
        __syncthreads();
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
    // r_ii = ||p|| and p^T e from one exchange
    double v2 = 0.0, pe = 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        v2 += p[r] * p[r];
        pe += p[r] * e[rlo + r];
    }
    v2 = qr_block_sum(v2, red4);
    pe = qr_block_sum(pe, red4);
    if (threadIdx.x == 0) {
        scal[0] = v2;
        scal[1] = pe;
    }
    cl.sync();
    const double rii = sqrt(qr_rank_sum(cl, scal, 0, nq));
    const double pet = qr_rank_sum(cl, scal, 1, nq);
    const double dmax = fmax(dmax0, rii);
    const double dmin = (i == 0) ? rii : fmin(dmin0, rii);
    const double kappa = (dmin > 0.0) ? dmax / dmin : INFINITY;
    if (!(kappa <= thr)) {  // C2 (also rii == 0 or NaN): drop column i, keep k = i
        if (q == 0 && threadIdx.x == 0) {
            cyc->stopped = 1;
            cyc->k = i;
            cyc->reason = (i == 0) ? 5 : 2;
        }
        cl.sync();  // no CTA leaves while another may still read its shared memory
        return;
    }
    const double inv = 1.0 / rii;
    const double di = pet * inv;
    double ee = 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const double qv = p[r] * inv;
        Q[(int64_t)i * s + rlo + r] = qv;
        const double ev = e[rlo + r] - di * qv;
        e[rlo + r] = ev;
        ee += ev * ev;
    }
    ee = qr_block_sum(ee, red4);
    if (threadIdx.x == 0) scal[2] = ee;
    cl.sync();
    const double rh = sqrt(qr_rank_sum(cl, scal, 2, nq));
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
// Per problem (one warp each): y = R_k^{-1} d by back substitution, coef_l = y_l * sigma_l.
__global__ void k_inner_ls(const Plan P) {
    extern __shared__ double rhs[];
    const int p = blockIdx.x, m = P.m;
    if (P.pflag[p] & 1) return;
    const double* R = P.R + (int64_t)p * m * m;
    const double* d = P.d + (int64_t)p * m;
    const double* sigma = P.sigma + (int64_t)p * (m + 1);
    double* y = P.y + (int64_t)p * m;
    double* coef = P.coef + (int64_t)p * m;
    const int k = P.cyc[p].k;
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
    if (p == 0 && P.gsync) {  // the fused step's grid counter and its give-up flag
        P.gsync[0] = 0;
        P.gsync[1] = 0;
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

template <int V, int U, int NW, typename MT, typename VT, typename AT>
static void inner_spmv_v(const Plan& p, int i, const MT* val) {
    const size_t sm = (size_t)(p.Bn + 1) * sizeof(AT);
    set_smem((const void*)k_inner_spmv<V, U, NW, MT, VT, AT>, sm);
    k_inner_spmv<V, U, NW, MT, VT, AT><<<p.nblk, 512, sm, p.st>>>(p, i, val);
}

template <int NW, typename MT, typename VT, typename AT>
static void inner_spmv_nw(const Plan& p, int i, const MT* val) {
    if (p.vec == 0) inner_spmv_v<0, 1, NW, MT, VT, AT>(p, i, val);
    else if (p.vec == 1) {
        if constexpr (sizeof(MT) == 8) {  // FP64 one thread per row reads the SELL-32 copy (always built for it)
            if (p.sl_off) inner_spmv_v<kVecSell, 1, NW, MT, VT, AT>(p, i, p.sl_val);
            else inner_spmv_v<8, 4, NW, MT, VT, AT>(p, i, val);
        } else {
            inner_spmv_v<1, 1, NW, MT, VT, AT>(p, i, val);
        }
    }
    else if (p.vec <= 8) inner_spmv_v<8, 4, NW, MT, VT, AT>(p, i, val);
    else inner_spmv_v<32, 2, NW, MT, VT, AT>(p, i, val);
}

template <int G, int NW, typename MT, typename VT, typename AT>
static void inner_spmv_g(const Plan& p, int i, const MT* val) {
    const size_t sm = (size_t)G * (p.Bn + 1) * sizeof(AT);
    set_smem((const void*)k_inner_spmv_grp<G, NW, MT, VT, AT>, sm);
    k_inner_spmv_grp<G, NW, MT, VT, AT><<<p.ngrp, 512, sm, p.st>>>(p, i, val);
}

template <int NW, typename MT, typename VT, typename AT>
static void inner_spmv_gsel(const Plan& p, int i, const MT* val) {
    if (p.G == 2) inner_spmv_g<2, NW, MT, VT, AT>(p, i, val);
    else inner_spmv_g<4, NW, MT, VT, AT>(p, i, val);
}

template <typename MT, typename VT, typename AT>
static void inner_spmv_t(const Plan& p, int i, const MT* val) {
    const int nwin = (p.t > 0) ? std::min(p.t, i + 1) : 0;
    if (p.G > 1) {  // grouped right-hand sides (one thread per row); windows above 4 are not grouped
        switch (nwin) {
            case 0: inner_spmv_gsel<0, MT, VT, AT>(p, i, val); return;
            case 1: inner_spmv_gsel<1, MT, VT, AT>(p, i, val); return;
            case 2: inner_spmv_gsel<2, MT, VT, AT>(p, i, val); return;
            case 3: inner_spmv_gsel<3, MT, VT, AT>(p, i, val); return;
            case 4: inner_spmv_gsel<4, MT, VT, AT>(p, i, val); return;
            default: break;
        }
    }
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

// ---- fused step ----
template <int V, int U, int NW, typename MT, typename VT, typename AT>
static bool inner_step_v(const Plan& p, int i, const MT* val, bool last) {
    const void* fn = (const void*)k_inner_step<V, U, NW, MT, VT, AT>;
    const size_t sm = (size_t)(p.Bn + 1) * sizeof(AT);
    set_smem(fn, sm);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 512, sm) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if ((int64_t)per_sm * p.sms < p.nblk) return false;  // not one wave: the two kernels
    k_inner_step<V, U, NW, MT, VT, AT><<<p.nblk, 512, sm, p.st>>>(p, i, val, last ? 1 : 0);
    return true;
}

template <int NW, typename MT, typename VT, typename AT>
static bool inner_step_nw(const Plan& p, int i, const MT* val, bool last) {
    if (p.vec == 0) {  // length-binned SpMV: fused in FP32 only (FP64 measured slower fused: 399 vs 380 ms, Zipf 2M)
        if constexpr (sizeof(MT) == 8) return false;
        else return inner_step_v<0, 1, NW, MT, VT, AT>(p, i, val, last);
    }
    if (p.vec == 1) {
        if constexpr (sizeof(MT) == 8) {  // FP64 one thread per row reads the SELL-32 copy
            return p.sl_off ? inner_step_v<kVecSell, 1, NW, MT, VT, AT>(p, i, p.sl_val, last) : false;
        } else {
            return inner_step_v<1, 1, NW, MT, VT, AT>(p, i, val, last);
        }
    }
    if (p.vec <= 8) return inner_step_v<8, 4, NW, MT, VT, AT>(p, i, val, last);
    return inner_step_v<32, 2, NW, MT, VT, AT>(p, i, val, last);
}

template <typename MT, typename VT, typename AT>
static bool inner_step_t(const Plan& p, int i, const MT* val, bool last) {
    const int nwin = (p.t > 0) ? std::min(p.t, i + 1) : 0;
    switch (nwin) {
        case 0: return inner_step_nw<0, MT, VT, AT>(p, i, val, last);
        case 1: return inner_step_nw<1, MT, VT, AT>(p, i, val, last);
        case 2: return inner_step_nw<2, MT, VT, AT>(p, i, val, last);
        case 3: return inner_step_nw<3, MT, VT, AT>(p, i, val, last);
        case 4: return inner_step_nw<4, MT, VT, AT>(p, i, val, last);
        default: return false;  // wider windows: the two kernels
    }
}

bool launch_inner_step(const Plan& p, int i, bool last) {
    if (p.G > 1 || !p.gsync) return false;
    bool ok;
    if (p.prec == kFP64) ok = inner_step_t<double, double, double>(p, i, p.val, last);
    else if (p.prec == kFP32) ok = inner_step_t<float, float, float>(p, i, p.val32, last);
    else ok = inner_step_t<float, __nv_bfloat16, float>(p, i, p.val32, last);
    if (ok) ++g_launches;
    return ok;
}

template <int NW, typename VT, typename AT>
static void inner_axpy_nw(const Plan& p, int i, bool last) {
    k_inner_axpy<NW, VT, AT><<<p.nblk, 512, 0, p.st>>>(p, i, last ? 1 : 0);
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
    const int nq = p.qr_cluster;
    const int nrmax = (p.s + nq - 1) / nq;
    const size_t sm = (size_t)(nrmax + 3 * p.m) * sizeof(double);
    set_smem((const void*)k_inner_qr, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nq * p.P), 1, 1);
    cfg.blockDim = dim3(128, 1, 1);
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
    k_inner_ls<<<p.P, 32, (size_t)p.m * sizeof(double), p.st>>>(p);
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
