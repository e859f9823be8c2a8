// CSR SpMV over one row block, result into shared memory (used by the inner and outer steps).
#pragma once

#include "common.cuh"

namespace sfg {

// out[r - r0] = scale * sum_p val[p] * x[col[p]] for rows r in [r0, r1).
// Each row is handled by a sub-warp of V lanes; a warp processes U sub-warp rows at once (all their loads issued
// before the FMAs) so every thread keeps several independent loads in flight.  For a fixed unroll slot the warp's
// sub-warps read consecutive rows, so the col/val streams are read in contiguous segments.  The per-row sums are
// combined by a fixed xor-shuffle tree, so the result does not depend on scheduling.
template <int V, int U, typename MT, typename XT, typename AT>
__device__ __forceinline__ void spmv_rows_to_smem(const int* __restrict__ rp, const int* __restrict__ col,
                                                  const MT* __restrict__ val, const XT* __restrict__ x, int r0,
                                                  int r1, AT scale, AT* __restrict__ out) {
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
            if (sl == 0 && row < r1) out[row - r0] = scale * sum[u];
        }
    }
}

// Dispatch on the sub-warp width chosen at run time (2..32); U is fixed per width.
#define SFG_SPMV_DISPATCH(V_RUNTIME, CALL)          \
    switch (V_RUNTIME) {                            \
        case 2: { constexpr int VV = 2, UU = 4; CALL; } break;   \
        case 4: { constexpr int VV = 4, UU = 4; CALL; } break;   \
        case 8: { constexpr int VV = 8, UU = 4; CALL; } break;   \
        case 16: { constexpr int VV = 16, UU = 2; CALL; } break; \
        default: { constexpr int VV = 32, UU = 2; CALL; } break; \
    }

}  // namespace sfg
