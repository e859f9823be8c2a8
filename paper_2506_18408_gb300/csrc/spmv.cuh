// CSR SpMV over one row block, result into shared memory (used by the inner and outer steps).
#pragma once

#include "common.cuh"

namespace sfg {

// CNT entries (compile-time count) of one row chunk: loads first, then exactly CNT FMAs.  Lanes whose row has
// fewer entries in this chunk are predicated off; the warp issues no instruction for slots no lane needs.
template <int CNT, typename MT, typename XT, typename AT>
__device__ __forceinline__ void row_chunk(const int* __restrict__ col, const MT* __restrict__ val,
                                          const XT* __restrict__ x, int a, int len, int pk, AT& sum) {
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
    for (int q = 0; q < CNT; ++q)
        if (pk + q < len) sum += v[q] * load_as(x + c[q], AT());
}

// out[r - r0] = sum_p val[p] * x[col[p]] for rows r in [r0, r1), one thread per row.
// Warps walk the rows together; each row is read in chunks of up to 4 entries whose count is the longest row of
// the warp in that chunk, dispatched to a compile-time count, so the number of FMA instructions a warp issues is
// exactly its longest row (with no shuffle tree): the FP64 pipe, scarce on this GPU, does only useful work.
// The next row group's extents are fetched while the current one is summed.  Sums run in entry order.
template <typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_rows_scalar(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const MT* __restrict__ val, const XT* __restrict__ x, int r0,
                                                 int r1, AT* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    int rw = r0 + (threadIdx.x & ~31);
    int a = 0, len = 0;
    if (rw + lane < r1) {
        a = __ldg(rp + rw + lane);
        len = __ldg(rp + rw + lane + 1) - a;
    }
    for (; rw < r1; rw += blockDim.x) {  // warp-uniform loop
        const int rn = rw + (int)blockDim.x + lane;
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
                case 4: row_chunk<4>(col, val, x, a, len, pk, sum); break;
                default: row_chunk<4>(col, val, x, a, len, pk, sum); break;
            }
        }
        if (rw + lane < r1) out[rw + lane - r0] = sum;
        a = an;
        len = lenn;
    }
}

// Same result with each row handled by a sub-warp of V lanes; a warp processes U sub-warp rows at once (all their
// loads issued before the FMAs).  For a fixed unroll slot the warp's sub-warps read consecutive rows, so the
// col/val streams are read in contiguous segments.  Per-row sums are combined by a fixed xor-shuffle tree.
// Suited to long or irregular rows.
template <int V, int U, typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_rows_vector(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const MT* __restrict__ val, const XT* __restrict__ x, int r0,
                                                 int r1, AT* __restrict__ out) {
    constexpr int SUBS = 32 / V;
    constexpr int TILE = SUBS * U;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int sub = lane / V, sl = lane % V;
    for (int tb = r0 + warp * TILE; tb < r1; tb += nwarps * TILE) {
        int beg[U], len[U];
        int maxlen = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int row = tb + u * SUBS + sub;
            if (row < r1) {
                beg[u] = __ldg(rp + row);
                len[u] = __ldg(rp + row + 1) - beg[u];
            } else {
                beg[u] = 0;
                len[u] = 0;
            }
            maxlen = max(maxlen, len[u]);
        }
        AT sum[U];
#pragma unroll
        for (int u = 0; u < U; ++u) sum[u] = AT(0);
        for (int p = sl; p < maxlen; p += V) {
            int c[U];
            AT v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (p < len[u]) {
                    c[u] = __ldg(col + beg[u] + p);
                    v[u] = (AT)__ldg(val + beg[u] + p);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (p < len[u]) sum[u] += v[u] * load_as(x + c[u], AT());
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int o = V / 2; o > 0; o >>= 1) sum[u] += __shfl_xor_sync(0xffffffffu, sum[u], o);
            const int row = tb + u * SUBS + sub;
            if (sl == 0 && row < r1) out[row - r0] = sum[u];
        }
    }
}

// Rows [lo, hi) of a block's length-sorted order (local offsets pm[i]), each handled by a sub-warp of V lanes, U rows
// per sub-warp at once, each lane taking E entries of a row per pass (all loads of a pass issued before its FMAs,
// so E * U gathers per lane are in flight); a lane's entries are p, p + V, p + 2V, ... in that order and the per-row
// sums are combined by a fixed xor-shuffle tree.
template <int V, int U, int E, typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_sorted_vector(const int* __restrict__ rpm, const int* __restrict__ col,
                                                   const MT* __restrict__ val, const XT* __restrict__ x,
                                                   const uint16_t* __restrict__ pm, int lo, int hi,
                                                   AT* __restrict__ out, const int* __restrict__ brpm) {
    constexpr int SUBS = 32 / V;
    constexpr int TILE = SUBS * U;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int sub = lane / V, sl = lane % V;
    for (int tb = lo + warp * TILE; tb < hi; tb += nwarps * TILE) {
        int beg[U], len[U], kk[U];
        int maxlen = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = tb + u * SUBS + sub;
            kk[u] = -1;
            beg[u] = 0;
            len[u] = 0;
            if (i < hi) {
                kk[u] = pm[i];
                const int* rq = brpm ? brpm + i : rpm + kk[u];  // the copy in processing order, or the CSR row
                beg[u] = __ldg(rq);
                len[u] = __ldg(rq + 1) - beg[u];
            }
            maxlen = max(maxlen, len[u]);
        }
        maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)maxlen);
        AT sum[U];
#pragma unroll
        for (int u = 0; u < U; ++u) sum[u] = AT(0);
        for (int p0 = sl; p0 < maxlen; p0 += E * V) {
            int c[U][E];
            AT v[U][E];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = p0 + e * V;
                    if (p < len[u]) {
                        c[u][e] = __ldg(col + beg[u] + p);
                        v[u][e] = (AT)__ldg(val + beg[u] + p);
                    }
                }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (p0 + e * V < len[u]) sum[u] += v[u][e] * load_as(x + c[u][e], AT());
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int o = V / 2; o > 0; o >>= 1) sum[u] += __shfl_xor_sync(0xffffffffu, sum[u], o);
            if (sl == 0 && kk[u] >= 0) out[kk[u]] = sum[u];
        }
    }
}

// Length-binned SpMV of one block for matrices with irregular rows: out[k] for the block's local rows k, matrix rows
// m0 + k.  The block's rows come in a precomputed order pm[0 .. len) (local offsets): first the rows with at most 16
// entries sorted by length (n0 of them), then rows of 17..64 entries (up to n01), then longer rows.  Short rows take
// one thread each: a warp's 32 rows have (nearly) the same length, so the compile-time chunk loop issues about as
// many FMAs as there are entries and 32 rows' loads are in flight per warp.  Medium rows take 8 lanes, long rows a
// whole warp.  Every row's sum still runs over its entries in a fixed order (per lane, then a fixed shuffle tree).
// With brp (the copy of the matrix that stores each block's rows in this order: row i at brp[m0 + i], col and val
// then being that copy's arrays) the rows processed together are neighbours in memory; without it the CSR rows are
// read through pm.
template <typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_rows_binned(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const MT* __restrict__ val, const XT* __restrict__ x, int m0, int len,
                                                 const uint16_t* __restrict__ perm, int n0, int n01,
                                                 AT* __restrict__ out, const int* __restrict__ brp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint16_t* pm = perm + m0;
    const int* rpm = rp + m0;
    const int* brpm = brp ? brp + m0 : nullptr;
    for (int i0 = warp * 32; i0 < n0; i0 += nwarps * 32) {  // warp-uniform loop over the short rows
        const int i = i0 + lane;
        int k = -1, a = 0, rl = 0;
        if (i < n0) {
            k = pm[i];
            const int* rq = brpm ? brpm + i : rpm + k;
            a = __ldg(rq);
            rl = __ldg(rq + 1) - a;
        }
        const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)rl);
        AT sum = AT(0);
        for (int pk = 0; pk < maxlen; pk += 4) {
            switch (min(maxlen - pk, 4)) {
                case 1: row_chunk<1>(col, val, x, a, rl, pk, sum); break;
                case 2: row_chunk<2>(col, val, x, a, rl, pk, sum); break;
                case 3: row_chunk<3>(col, val, x, a, rl, pk, sum); break;
                default: row_chunk<4>(col, val, x, a, rl, pk, sum); break;
            }
        }
        if (k >= 0) out[k] = sum;
    }
    spmv_sorted_vector<8, 2, 2, MT, XT, AT>(rpm, col, val, x, pm, n0, n01, out, brpm);
    spmv_sorted_vector<32, 2, 4, MT, XT, AT>(rpm, col, val, x, pm, n01, len, out, brpm);
}

// V == 0: length-binned (perm, n0, n01, brp as for spmv_rows_binned); V == 1: one thread per row; else V lanes per
// row.
template <int V, int U, typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_rows_to_smem(const int* __restrict__ rp, const int* __restrict__ col,
                                                  const MT* __restrict__ val, const XT* __restrict__ x, int r0,
                                                  int r1, AT* __restrict__ out, const uint16_t* perm = nullptr,
                                                  int n0 = 0, int n01 = 0, const int* brp = nullptr) {
    if constexpr (V == 0) spmv_rows_binned<MT, XT, AT>(rp, col, val, x, r0, r1 - r0, perm, n0, n01, out, brp);
    else if constexpr (V == 1) spmv_rows_scalar<MT, XT, AT>(rp, col, val, x, r0, r1, out);
    else spmv_rows_vector<V, U, MT, XT, AT>(rp, col, val, x, r0, r1, out);
}

// Dispatch on the lanes-per-row width chosen at run time (0 = length-binned, 1 = one thread per row, else 2..32).
#define SFG_SPMV_DISPATCH(V_RUNTIME, CALL)                       \
    switch (V_RUNTIME) {                                         \
        case 0: { constexpr int VV = 0, UU = 1; CALL; } break;   \
        case 1: { constexpr int VV = 1, UU = 1; CALL; } break;   \
        case 2: { constexpr int VV = 2, UU = 4; CALL; } break;   \
        case 4: { constexpr int VV = 4, UU = 4; CALL; } break;   \
        case 8: { constexpr int VV = 8, UU = 4; CALL; } break;   \
        case 16: { constexpr int VV = 16, UU = 2; CALL; } break; \
        default: { constexpr int VV = 32, UU = 2; CALL; } break; \
    }

}  // namespace sfg
