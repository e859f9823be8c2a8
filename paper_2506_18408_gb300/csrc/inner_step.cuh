// Kernels of one inner step of a sketched-GMRES cycle (Section 3, Section 4.1) -- the fused inner SpMV (w' = A u_i,
// truncated-Arnoldi window dots, ||u_i||^2, per-block sketch partials), the truncated-Arnoldi update and the fused
// step that runs both in one launch -- as templates over the SpMV shape, the window size and the precision, with
// their launch dispatch.  inner_f64.cu, inner_f32.cu and inner_bf16.cu instantiate them per precision (so they compile
// in parallel); inner.cu holds the rest of the cycle.
#pragma once

#include "kernels.h"
#include "spmv.cuh"

#include <climits>
#include <algorithm>

namespace sfg {

// Template value of k_inner_spmv's lanes-per-row parameter for one thread per row reading the SELL-32 copy of A
// (the FP64 inner cycle); 1 is one thread per row reading the CSR arrays.
constexpr int kVecSell = -1;

__device__ __forceinline__ bool cycle_idle(const Plan& P, int p, int i) {
    const CycleState* c = P.cyc + p;
    return c->stopped || c->brk_step <= i || (P.pflag[p] & 1);
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// The one-thread-per-row SpMVs request into L2, this many row groups (CTA-wide rounds of rows) ahead, the line of x
// that holds each row's own entry (the diagonal's column).  A block's first rows are otherwise first fetched from
// HBM by the row's own gather (no earlier block has touched them: with a banded matrix the rows of the block below
// read them only as their far band, later in the launch), so the lines come in a round trip later than the rest.
// One group ahead measured best (128^3 FP64 solve: 46.0 ms, against 46.7 ms two groups and 46.8 ms three ahead).
constexpr int kXPrefetchAhead = 1;

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
// storing w' (global W and the shared block copy) and the window dot products acc_q += u_{lo+q}[r] * w'[r].  Each
// row is summed in entry order, the warp issuing as many FMAs as its slice is wide.  The window values and the next
// slice's extent are loaded before the row's SpMV, so they are in flight together.  Returns the thread's largest
// exponent of w'.
template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ int spmv_dots_sell(int N, const int* __restrict__ soff, const uint8_t* __restrict__ slen,
                                              const int* __restrict__ scol, const MT* __restrict__ sval, int sb,
                                              const VT* __restrict__ Ub, const VT* __restrict__ xg, int i, int lo,
                                              int v0, int len, int cs, AT* __restrict__ wblk, AT* __restrict__ W,
                                              AT (&acc)[NW > 0 ? NW : 1]) {
    const int lane = threadIdx.x & 31;
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    const VT* xs = xg + cs;  // gather base (u_i, or M^{-1} u_i with a preconditioner): column c at vector index c + cs
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
        const int kn = kw + (int)blockDim.x;
        int o0n = 0, o1n = 0, rln = 0;
        if (kn < len) {
            const int sid = sb + (kn >> 5);
            o0n = __ldg(soff + sid);
            o1n = __ldg(soff + sid + 1);
            rln = __ldg(slen + (int64_t)sid * 32 + lane);
        }
        const int kp = k + kXPrefetchAhead * (int)blockDim.x;
        if (kp < len) prefetch_l2(xg + v0 + kp);  // x of the row's own column, kXPrefetchAhead row group(s) ahead
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
        emax = max(emax, exp_of(sum));
        o0 = o0n;
        o1 = o1n;
        rl = rln;
    }
    return emax;
}

// ---------------------------------------------------------------------------------------------------------------
// Phase 1, one thread per row: w' = A u_i over the block (vector rows v0 .. v0+len = matrix rows v0-cs ..) fused
// with storing w' (global W and the shared block copy) and the window dot products acc_q += u_{lo+q}[r] * w'[r].
// The window values and the next row group's extents are loaded before the row's SpMV, so they are in flight
// together.  Returns the thread's largest exponent of w'.
template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ int spmv_dots_scalar(int N, const int* __restrict__ rp, const int* __restrict__ col,
                                                const MT* __restrict__ val, const VT* __restrict__ Ub,
                                                const VT* __restrict__ xg, int i, int lo, int v0, int len, int cs,
                                                AT* __restrict__ wblk, AT* __restrict__ W,
                                                AT (&acc)[NW > 0 ? NW : 1]) {
    const int lane = threadIdx.x & 31;
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    const VT* xs = xg + cs;               // gather base (u_i, or M^{-1} u_i): column c at vector index c + cs
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
        const int kn = k + (int)blockDim.x;
        int an = 0, rln = 0;
        if (kn < len) {
            an = __ldg(rpm + kn);
            rln = __ldg(rpm + kn + 1) - an;
        }
        const int kp = k + kXPrefetchAhead * (int)blockDim.x;
        if (kp < len) prefetch_l2(xg + v0 + kp);  // x of the row's own column, kXPrefetchAhead row group(s) ahead
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
        emax = max(emax, exp_of(sum));
        a = an;
        rl = rln;
    }
    return emax;
}

// Phase 1 tail for the sub-warp path (w' already in shared memory): store w' and accumulate the window dots.
template <int NW, typename VT, typename AT>
__device__ __forceinline__ int dots_pass(int N, int v0, int len, const VT* __restrict__ Ub, int lo,
                                         const AT* __restrict__ wblk, AT* __restrict__ W,
                                         AT (&acc)[NW > 0 ? NW : 1]) {
    const unsigned long long pol = l2_keep_policy();  // window rows and w' are read again by the update
    int emax = 1;
#pragma unroll 2
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const int r = v0 + k;
        const AT w = wblk[k];
        st_keep(W + r, w, pol);
        emax = max(emax, exp_of(w));
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += ld_keep(Ub + (int64_t)(lo + q) * N + r, pol) * w;
    }
    return emax;
}

// ---------------------------------------------------------------------------------------------------------------
// Phase 1 of an inner step for the CTA's row block: w' = A u_i (stored to W and kept in the shared block), the
// block partials of the window dots (hpart), and Eb, the block's largest exponent of w' (the reference exponent of
// the FP64 fixed-point sketch sums).  (The block partials of ||u_i||^2 come from the update that wrote u_i.)  Returns false (every thread of the CTA alike) when
// the block's problem has no step i to take.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ bool inner_spmv_part(const Plan& P, int i, const MT* __restrict__ val,
                                                AT* __restrict__ wblk, int& Eb) {
    __shared__ AT red[512];
    __shared__ int stop_sh, emax_sh[16];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    if (threadIdx.x == 0) stop_sh = cycle_idle(P, bi.prob, i) ? 1 : 0;
    __syncthreads();
    if (stop_sh) return false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Bn = P.Bn, N = P.N;
    const VT* Ub = (const VT*)P.U;
    AT* W = (AT*)P.W;
    const int lo = i - NW + 1;  // window u_lo..u_i (NW = min(t, i+1))
    AT acc[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) acc[q] = AT(0);
    int emax;
    // the vector the SpMV multiplies: u_i, or t_i = M^{-1} u_i with a right preconditioner (an FP64 plan only)
    const VT* xg = P.xin ? reinterpret_cast<const VT*>(P.xin) : Ub + (int64_t)i * N;
    if constexpr (V == kVecSell) {
        emax = spmv_dots_sell<NW>(N, P.sl_off, P.sl_len, P.sl_col, val, P.sl_base[bi.list], Ub, xg, i, lo, bi.v0,
                                  bi.len, bi.cs, wblk, W, acc);
    } else if constexpr (V == 1) {
        emax = spmv_dots_scalar<NW>(N, P.rp, P.col, val, Ub, xg, i, lo, bi.v0, bi.len, bi.cs, wblk, W, acc);
    } else {
        const int m0 = bi.v0 - bi.cs;
        int n0, n01;
        block_bins(P, bi, n0, n01);
        if constexpr (V == 0 && sizeof(MT) == 8) {  // FP64: the copy that stores the block's rows in this order
            if (P.brp) {
                spmv_rows_to_smem<V, U, MT, VT, AT>(P.rp, P.bcol, reinterpret_cast<const MT*>(P.bval), xg + bi.cs,
                                                    m0, m0 + bi.len, wblk, P.perm, n0, n01, P.brp);
            } else {
                spmv_rows_to_smem<V, U, MT, VT, AT>(P.rp, P.col, val, xg + bi.cs, m0, m0 + bi.len, wblk, P.perm, n0,
                                                    n01);
            }
        } else {
            spmv_rows_to_smem<V, U, MT, VT, AT>(P.rp, P.col, val, xg + bi.cs, m0, m0 + bi.len, wblk, P.perm, n0,
                                                n01);
        }
        __syncthreads();
        emax = dots_pass<NW>(N, bi.v0, bi.len, Ub, lo, wblk, W, acc);
    }
    if (threadIdx.x == 0) wblk[Bn] = AT(0);
    // block sums of the window dots in one round: each warp's sums (shuffle trees), then the warps' partials in
    // warp order; the block's largest exponent of w' with them
    {
        AT (*red2)[16] = reinterpret_cast<AT (*)[16]>(red);  // [NW][16]
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const AT d = warp_sum(acc[q]);
            if (lane == 0) red2[q][warp] = d;
        }
        emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
        if (lane == 0) emax_sh[warp] = emax;
        __syncthreads();
        if ((int)threadIdx.x < NW) {
            AT t = AT(0);
            for (int w = 0; w < nw; ++w) t += red2[threadIdx.x][w];
            ((AT*)P.hpart)[(int64_t)b * kMaxTrunc + threadIdx.x] = t;
        }
    }
    Eb = 1;
    for (int q = 0; q < nw; ++q) Eb = max(Eb, emax_sh[q]);
    return true;
}

// Prepares the shared block of w' for the sketch gathers: FP64, converted in place to its 64-bit fixed-point image
// relative to 2^Eb (exact integer sums, independent of order; the FP64 pipe stays with the SpMV), with the zero slot
// at Bn; FP32, as it is.  Ends with a block barrier.
template <typename AT>
__device__ __forceinline__ void sketch_prepare(const Plan& P, int len, AT* __restrict__ wblk, int Eb) {
    if constexpr (sizeof(AT) == 8) {
        const int H = P.sk_headroom;
        long long* qblk = reinterpret_cast<long long*>(wblk);
        for (int r = threadIdx.x; r <= P.Bn; r += blockDim.x) qblk[r] = (r < len) ? to_fixed((double)wblk[r], Eb, H) : 0;
    }
    __syncthreads();
}

// Per-block sketch partials of w' for sketch rows r0, r0 + rstep, ... < s: cpart[b*s + r] = sum over the block's list
// for row r (in list order) of +-w'.  FP64: from the fixed-point image, converted to FP64 once per row.
template <typename AT>
__device__ __forceinline__ void sketch_rows(const Plan& P, int b, int list, const AT* __restrict__ wblk, int Eb, int r0,
                                            int rstep) {
    const int s = P.s, ng = (s + 31) / 32;
    const int* sg = P.seg + (int64_t)list * ng;  // the block's group starts (units)
    AT* cpart = (AT*)P.cpart;
    if constexpr (sizeof(AT) == 8) {
        const long long* qblk = reinterpret_cast<const long long*>(wblk);
        const double unit = fixed_unit(0.0, Eb, P.sk_headroom);
        const bool bad = exp_nonfinite(0.0, Eb);
        for (int rr = r0; rr < s; rr += rstep) {
            const int g = rr >> 5;
            const long long v = sum_group(P.ent, sg[g], (sg[g + 1] - sg[g]) >> 5, rr & 31, qblk);
            cpart[(int64_t)b * s + rr] = bad ? (AT)NAN : (AT)((double)v * unit);
        }
    } else {
        for (int rr = r0; rr < s; rr += rstep) {
            const int g = rr >> 5;
            cpart[(int64_t)b * s + rr] = sum_group(P.ent, sg[g], (sg[g + 1] - sg[g]) >> 5, rr & 31, wblk);
        }
    }
}

// The inner SpMV kernel of the two-launch step: phase 1, then the block's sketch partials for every sketch row.
// Shared memory: the block of w' (Bn + 1 slots of AT, slot Bn = 0 for the list padding).
// At most 56 registers per thread (registers are allocated in units of 8 per thread): two 512-thread CTAs per SM
// then leave room for the sketched-QR cluster's CTAs to run beside them instead of displacing them.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(56) k_inner_spmv(const Plan P, int i, const MT* __restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    int Eb = 1;
    if (!inner_spmv_part<V, U, NW, MT, VT, AT>(P, i, val, wblk, Eb)) return;
    const int b = blockIdx.x;
    sketch_prepare(P, P.blk_len[b], wblk, Eb);
    sketch_rows(P, b, P.blk_list[b], wblk, Eb, threadIdx.x, blockDim.x);
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

// The truncated-Arnoldi update of a row block works on 64-row chunks (lane l of a warp: rows 64c + l and 64c + 32 + l)
// and forms the block partial of ||u_{i+1}||^2 on the way: each lane accumulates the squares of the stored values of
// its rows in the order of its chunks (one FMA per row), the block partial is the warps' shuffle-tree sums added in
// warp order.  Warp w takes chunks w, w + nw, w + 2 nw, ... in both the two-launch update and the fused step, so
// the two compute the same sums in the same order.  The norm partials alternate between two slots by step parity:
// step i reads slot i & 1 (written by the update of step i - 1) and writes the other.
__host__ __device__ constexpr int norm_chunks(int rows) { return (rows + 63) / 64; }

// Truncated-Arnoldi update kernel of the two-launch step (NW = window size).  Warp w updates the 64-row chunks w,
// w + nw, ... of the block (lane l: rows 64c + l and 64c + 32 + l) and its first chunk's rows of w' and of the window
// vectors are loaded first (they do not depend on the scalars); meanwhile warp 0 sums the problem's ||u_i||^2
// partials and warps 1..NW its window-dot partials, each with all loads in flight at once.  After one barrier thread
// 0 forms sigma_i and the coefficients; after a second, the sketched column S A b_i (one warp per sketch row, rows
// spread over all of the problem's blocks) and the row update with the block partial of ||u_{i+1}||^2.
// Three 512-thread CTAs per SM (at most 42 registers; batches run many waves of blocks) for windows up to 3, two
// for wider windows, which would spill within 42.
template <int NW, typename VT, typename AT>
__device__ __forceinline__ void inner_axpy_block(const Plan& P, int i, int last) {
    __shared__ AT coef_sh[kMaxTrunc];
    __shared__ AT part_sh[32];  // [0..NW] the problem's sums; later the warps' norm sums
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
    AT wv[2], uv[2][NW > 0 ? NW : 1];
    // last reads of w' and of the oldest window vector (the next step's window starts one later): L2 may drop them
    // (FP64 and FP32 bases; measured slower with a BF16 basis, which keeps plain loads)
    constexpr bool DROP = sizeof(VT) >= 4;
    const unsigned long long drop = l2_drop_policy();
    auto win = [&](int q, int r) -> AT {
        const VT* a = Ub + (int64_t)(lo + q) * N + r;
        return (DROP && q == 0 && NW > 1) ? ld_keep(a, drop) : ld_plain(a);
    };
    auto wrd = [&](int r) -> AT { return DROP ? ld_keep(W + r, drop) : W[r]; };
    // the rows of chunk c for this lane, with their w' and window values
    auto load_chunk = [&](int c, AT (&w)[2], AT (&uq)[2][NW > 0 ? NW : 1]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int k = 64 * c + 32 * u + lane;
            const bool ok = k < bi.len;
            const int r = bi.v0 + k;
            w[u] = ok ? wrd(r) : AT(0);
#pragma unroll
            for (int q = 0; q < NW; ++q) uq[u][q] = ok ? win(q, r) : AT(0);
        }
    };
    if (!last) load_chunk(warp, wv, uv);
    if (threadIdx.x == 0) stop_sh = cycle_idle(P, p, i) ? 1 : 0;
    const int b0 = P.prob_b0[p], b1 = P.prob_b0[p + 1];
    // ||u_i||^2 (warp 0; sigma_0 is known at i = 0) and the window dots u_l^T w' (warp 1 + q) over the blocks
    if (warp == 0 && i > 0) {
        const AT a = block_partials_sum((const AT*)P.normpart + (int64_t)(i & 1) * P.nblk, 1, b0, b1, lane);
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
    AT nsq = AT(0);  // the lane's part of ||u_{i+1}||^2
    // updates the lane's rows of chunk c
    auto update_chunk = [&](int c, const AT (&w)[2], const AT (&uq)[2][NW > 0 ? NW : 1]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int k = 64 * c + 32 * u + lane;
            if (k < bi.len) {
                AT v = w[u];
#pragma unroll
                for (int q = 0; q < NW; ++q) v -= cf[q] * uq[u][q];
                if constexpr (sizeof(AT) == 8) v = mul_pow2((double)v, p2);
                else v = v * sc2;
                st_keep(un + bi.v0 + k, v, pol);  // the next step gathers it and reads it as a window row
                const AT vs = stored_value(v, un);
                nsq = fma_as(vs, vs, nsq);
            }
        }
    };
    const int nch = norm_chunks(bi.len);
    if (warp < nch) update_chunk(warp, wv, uv);
    for (int c = warp + nw; c < nch; c += nw) {
        AT wr[2], uq[2][NW > 0 ? NW : 1];
        load_chunk(c, wr, uq);
        update_chunk(c, wr, uq);
    }
    // block partial of ||u_{i+1}||^2 into the slot of step i + 1
    const AT ws = warp_sum(nsq);
    if (lane == 0) part_sh[warp] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
        AT t = AT(0);
        for (int w = 0; w < nw; ++w) t += part_sh[w];
        ((AT*)P.normpart)[(int64_t)((i + 1) & 1) * P.nblk + b] = t;
    }
}

template <int NW, typename VT, typename AT>
__global__ void __launch_bounds__(512, (NW <= 3) ? 3 : 2) k_inner_axpy(const Plan P, int i, int last) {
    inner_axpy_block<NW, VT, AT>(P, i, last);
}

// ---------------------------------------------------------------------------------------------------------------
// Named barrier among the first `threads` threads of the CTA (barrier 0 is __syncthreads).
__device__ __forceinline__ void bar_sync_named(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Bounded wait of one lane for a shared-memory flag set by another warp of the CTA; false if it gave up.
constexpr int kFlagPolls = 1 << 26;  // several seconds: well beyond the grid wait's own bound (the flag is set once that wait ends)
__device__ __forceinline__ bool wait_flag(const int* flag) {
    for (int it = 0; it < kFlagPolls; ++it) {
        if (*(const volatile int*)flag) return true;
        __nanosleep(64);
    }
    return false;
}

// Phase 2 of the fused step (after the CTA's grid-wide arrival), with the warps split by role so that the sketch
// gathers (shared memory and integer adds) run beside the row update (HBM):
//  * warps 0..NW: thread 0 waits for every CTA's phase-1 partials (grid counter 0); warp 0 sums the problem's
//    ||u_i||^2 partials and warps 1..NW its window-dot partials; thread 0 forms sigma_i and the coefficients and
//    publishes them through a shared-memory flag;
//  * the other warps: the block's sketch partials (every sketch row), then one arrival per CTA on grid counter 2;
//  * then every warp updates its 64-row chunks of the block (those of the two-launch update; the first round's
//    loads are issued before the first wait for the coefficients) and forms its part of ||u_{i+1}||^2; the last warp
//    through the update adds the warps' parts into the block's partial;
//  * last, the warps that own a row of the sketched column S A b_i (rows spread over all blocks) wait for every CTA's
//    sketch partials (grid counter 2) and sum them.
// The arithmetic of every value and its order are those of the two-launch step.
template <int NW, typename VT, typename AT>
__device__ __forceinline__ void fused_phase2(const Plan& P, int i, int last, AT* __restrict__ wblk, int Eb,
                                             const unsigned long long* target_ptr) {
    constexpr int NSW = NW + 1;  // warps of the scalar role
    constexpr bool WIDE = (sizeof(AT) == 8 && NW >= 3);
    __shared__ AT coef_sh[kMaxTrunc];
    __shared__ AT part_sh[kMaxTrunc + 1];
    __shared__ double sig_sh;
    __shared__ AT nrm_sh[32];
    __shared__ int stop_sh, ready_sh, skdone_sh, upd_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    const int p = bi.prob;
    if (threadIdx.x == 0) {
        stop_sh = 0;
        ready_sh = 0;
        skdone_sh = 0;
        upd_sh = 0;
    }
    sketch_prepare(P, bi.len, wblk, Eb);  // ends with a block barrier: the flags above and *target_ptr are visible
    const unsigned long long target = *target_ptr;
    const int N = P.N, s = P.s, m = P.m;
    const int b0 = P.prob_b0[p], b1 = P.prob_b0[p + 1];
    const int lo = i - NW + 1;
    if (warp < NSW) {
        if (threadIdx.x == 0) grid_wait(P.gsync, target, P.gsync + 1);
        bar_sync_named(1, NSW * 32);
        if (warp == 0 && i > 0) {
            const AT a = block_partials_sum((const AT*)P.normpart + (int64_t)(i & 1) * P.nblk, 1, b0, b1, lane);
            if (lane == 0) part_sh[0] = a;
        } else if (warp >= 1) {
            const AT a = block_partials_sum((const AT*)P.hpart + (warp - 1), kMaxTrunc, b0, b1, lane);
            if (lane == 0) part_sh[warp] = a;
        }
        bar_sync_named(1, NSW * 32);
        if (threadIdx.x == 0) {
            const bool lead = (b == b0);  // the problem's first block writes its scalars
            double* sigma = P.sigma + (int64_t)p * (m + 1);
            int stop = cycle_idle(P, p, i) ? 1 : 0;
            double sig = 1.0;
            if (!stop) {
                // sigma_i = 1/||u_i||
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
                if (bad) {
                    stop = 1;
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
            sig_sh = sig;
            stop_sh = stop;
            __threadfence_block();
            *(volatile int*)&ready_sh = 1;
        }
    } else {
        sketch_rows(P, b, bi.list, wblk, Eb, threadIdx.x - NSW * 32, (int)blockDim.x - NSW * 32);
        __threadfence();  // this warp's partials are visible device-wide before the CTA's arrival on counter 2
        __syncwarp();
        if (lane == 0 && atomicAdd(&skdone_sh, 1) == nw - NSW - 1) {
            __threadfence();
            atomicAdd(P.gsync + 2, 1ull);
        }
    }
    // the scalars, once per warp
    bool stop = false;
    double sig_i = 1.0;
    AT cf[NW > 0 ? NW : 1];
    auto get_scalars = [&]() {
        bool ok = true;
        if (lane == 0) {
            ok = wait_flag(&ready_sh);
            if (!ok) atomicOr(P.gsync + 1, 1ull);  // the solve reports the give-up; this warp writes nothing
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        __threadfence_block();
        stop = !ok || stop_sh;
        sig_i = sig_sh;
#pragma unroll
        for (int q = 0; q < NW; ++q) cf[q] = coef_sh[q];
    };
    bool have = false;
    AT nsq = AT(0);  // the lane's part of ||u_{i+1}||^2
    if (!last) {
        // u_{i+1} = 2^p2 (w' - sum_q coef_q u_{lo+q}), 2^p2 the power of two just below sigma_i, over the chunks of
        // the two-launch update (warp w: 64-row chunks w, w + nw, ...), CPI of them per round with all loads issued
        // first
        constexpr int CPI = WIDE ? 1 : 2;
        const int nch = norm_chunks(bi.len);
        const int cfirst = warp, cstep = nw, cend = nch;
        VT* Ub = (VT*)P.U;
        const AT* W = (const AT*)P.W;
        VT* un = Ub + (int64_t)(i + 1) * N;
        const unsigned long long keep = l2_keep_policy();
        // last reads of w' and of the oldest window vector (the next step's window starts one later): L2 may drop
        // them (FP64 and FP32 bases; a BF16 basis keeps plain loads)
        constexpr bool DROP = sizeof(VT) >= 4;
        const unsigned long long drop = l2_drop_policy();
        int p2 = 0;
        AT sc2 = AT(1);
        for (int c0 = cfirst; c0 < cend; c0 += CPI * cstep) {
            AT wr[CPI][2], uq[CPI][2][NW > 0 ? NW : 1];
#pragma unroll
            for (int j = 0; j < CPI; ++j) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int c = c0 + j * cstep;
                    const int k = 64 * c + 32 * u + lane;
                    const bool ok = c < cend && k < bi.len;
                    const int r = bi.v0 + k;
                    if constexpr (sizeof(AT) == 8) wr[j][u] = ok ? (DROP ? ld_keep(W + r, drop) : W[r]) : AT(0);
                    else wr[j][u] = ok ? wblk[k] : AT(0);  // FP32: w' is still the shared block
#pragma unroll
                    for (int q = 0; q < NW; ++q) {
                        const VT* ap = Ub + (int64_t)(lo + q) * N + r;
                        uq[j][u][q] = ok ? ((DROP && q == 0 && NW > 1) ? ld_keep(ap, drop) : ld_plain(ap)) : AT(0);
                    }
                }
            }
            if (!have) {
                get_scalars();
                have = true;
                if (stop) break;
                frexp(sig_i, &p2);  // sigma_i = f * 2^p2, f in [0.5, 1)
                p2 -= 1;
                sc2 = (AT)ldexp(1.0, p2);
            }
#pragma unroll
            for (int j = 0; j < CPI; ++j) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int c = c0 + j * cstep;
                    const int k = 64 * c + 32 * u + lane;
                    if (c < cend && k < bi.len) {
                        AT v = wr[j][u];
#pragma unroll
                        for (int q = 0; q < NW; ++q) v -= cf[q] * uq[j][u][q];
                        if constexpr (sizeof(AT) == 8) v = mul_pow2((double)v, p2);
                        else v = v * sc2;
                        st_keep(un + bi.v0 + k, v, keep);  // the next step gathers it and reads it as a window row
                        const AT vs = stored_value(v, un);
                        nsq = fma_as(vs, vs, nsq);
                    }
                }
            }
        }
    }
    if (!have) get_scalars();
    if (stop) return;
    if (!last) {
        // the block partial of ||u_{i+1}||^2: the warps' sums in warp order, added by the last warp through the update
        const AT ws = warp_sum(nsq);
        int fin = 0;
        if (lane == 0) {
            nrm_sh[warp] = ws;
            __threadfence_block();
            fin = (atomicAdd(&upd_sh, 1) == nw - 1) ? 1 : 0;
            if (fin) {
                __threadfence_block();
                AT t = AT(0);
                for (int w = 0; w < nw; ++w) t += nrm_sh[w];
                ((AT*)P.normpart)[(int64_t)((i + 1) & 1) * P.nblk + b] = t;
            }
        }
        __syncwarp();
    }
    // sketched column S A b_i = sigma_i S w': sketch row rr to warp nw - 1 - rr / nb of the problem's block rr % nb,
    // once every CTA's sketch partials are in place (the last warps first: with few rows per block the update's
    // chunks fall to the first warps)
    const double csc = P.sk_scale * sig_i;
    const int nb = b1 - b0;
    bool waited = false;
    for (int rr = (nw - 1 - warp) * nb + (b - b0); rr < s; rr += nw * nb) {
        if (!waited) {
            if (lane == 0) grid_wait(P.gsync + 2, target, P.gsync + 1);
            __syncwarp();
            waited = true;
        }
        const AT a = block_partials_sum((const AT*)P.cpart + rr, s, b0, b1, lane);
        if (lane == 0) P.C[((int64_t)p * m + i) * s + rr] = csc * (double)a;
    }
}

// One inner step in one launch, for plans whose row blocks all fit on the GPU at once (one wave): phase 1 (SpMV,
// window dots, ||u_i||^2), a grid-wide arrival of every CTA (also one with no step to take) on grid counter 0, then
// phase 2 (fused_phase2: the sketch partials beside the truncated-Arnoldi update, and the sketched column after a
// second grid-wide arrival, on counter 2).  Every CTA of the launch is resident at the same time (the host launches
// it only when the occupancy allows all blocks at once, beside the sketched-QR cluster), so the waits end; each
// gives up after a bounded number of polls and raises the plan's sync flag, which the outer step turns into an error.
template <int V, int U, int NW, typename MT, typename VT, typename AT>
__global__ void __maxnreg__(56) k_inner_step(const Plan P, int i, const MT* __restrict__ val, int last) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    __shared__ unsigned long long target_sh;
    int Eb = 1;
    const bool active = inner_spmv_part<V, U, NW, MT, VT, AT>(P, i, val, wblk, Eb);
    __threadfence();  // this thread's partials are visible device-wide before the CTA arrives
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long old = atomicAdd(P.gsync, 1ull);
        target_sh = (old / gridDim.x + 1) * (unsigned long long)gridDim.x + (unsigned long long)P.gwait_extra;
        if (!active) atomicAdd(P.gsync + 2, 1ull);  // no sketch partials from this CTA either
    }
    if (!active) return;
    fused_phase2<NW, VT, AT>(P, i, last, wblk, Eb, &target_sh);
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
    if (p.vec == 0) {  // length-binned SpMV: fused in FP32 only (FP64 measured slower fused: 353 vs 334 ms, Zipf 2M)
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

}  // namespace sfg
