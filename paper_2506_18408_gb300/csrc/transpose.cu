// Transpose of the CSR matrix (for the adjoint solve A^T x = b) and the pattern gradient used by differentiation.
//
// The transpose is built once on the device: column counts, their prefix sum, a counting fill, then a sort of each
// transposed row by original row index (ties by source position), so the layout -- and hence every sum formed from
// it -- is deterministic.  The source position of every transposed entry is kept, so new values of A are carried
// over by a gather without rebuilding the structure.
#include "kernels.h"

#include <algorithm>

namespace sfg {

__global__ void k_count_cols(int64_t nnz, const int* __restrict__ col, int* __restrict__ counts) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + col[p], 1);
}

// Exclusive prefix sum of counts[0..len) into out[0..len] (single block).
__global__ void k_scan_plain(const int* __restrict__ counts, int* __restrict__ out, int len) {
    __shared__ int sums[1024];
    const int tid = threadIdx.x, T = blockDim.x;
    const int chunk = (len + T - 1) / T;
    const int a = min(len, tid * chunk), bnd = min(len, a + chunk);
    int local = 0;
    for (int i = a; i < bnd; ++i) local += counts[i];
    sums[tid] = local;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int v = (tid >= off) ? sums[tid - off] : 0;
        __syncthreads();
        sums[tid] += v;
        __syncthreads();
    }
    int run = sums[tid] - local;
    for (int i = a; i < bnd; ++i) {
        out[i] = run;
        run += counts[i];
    }
    if (tid == T - 1) out[len] = sums[T - 1];
}

__global__ void k_fill_transpose(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const int* __restrict__ rpT, int* __restrict__ cursor, int* __restrict__ colT,
                                 int* __restrict__ srcT) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int p = rp[r]; p < rp[r + 1]; ++p) {
        const int c = col[p];
        const int pos = rpT[c] + atomicAdd(cursor + c, 1);
        colT[pos] = r;
        srcT[pos] = p;
    }
}

// Insertion sort of each transposed row by (original row, source position); rows are short.
__global__ void k_sort_rows(int n, const int* __restrict__ rpT, int* __restrict__ colT, int* __restrict__ srcT,
                            int* __restrict__ maxlen) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int a = rpT[r], e = rpT[r + 1];
    for (int i = a + 1; i < e; ++i) {
        const int c = colT[i], sidx = srcT[i];
        int j = i - 1;
        while (j >= a && (colT[j] > c || (colT[j] == c && srcT[j] > sidx))) {
            colT[j + 1] = colT[j];
            srcT[j + 1] = srcT[j];
            --j;
        }
        colT[j + 1] = c;
        srcT[j + 1] = sidx;
    }
    atomicMax(maxlen, e - a);
}

__global__ void k_gather_vals(int64_t nnz, const int* __restrict__ src, const double* __restrict__ val,
                              double* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = val[src[q]];
}

void launch_transpose(int n, int64_t nnz, const int* rp, const int* col, int* counts, int* rpT, int* colT,
                      int* srcT, int* maxlen, cudaStream_t st) {
    const int g = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_count_cols<<<std::max(g, 1), 256, 0, st>>>(nnz, col, counts);
    k_scan_plain<<<1, 1024, 0, st>>>(counts, rpT, n);
    cudaMemsetAsync(counts, 0, (size_t)n * sizeof(int), st);
    k_fill_transpose<<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, rpT, counts, colT, srcT);
    k_sort_rows<<<(n + 255) / 256, 256, 0, st>>>(n, rpT, colT, srcT, maxlen);
    g_launches += 4;
}

void launch_gather_vals(int64_t nnz, const int* src, const double* val, double* out, cudaStream_t st) {
    const int g = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_gather_vals<<<std::max(g, 1), 256, 0, st>>>(nnz, src, val, out);
    ++g_launches;
}

// out[p] += alpha * u[row(p)] * v[col(p)] over the stored entries (one thread per row, entries in order).
__global__ void k_pattern_outer(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ u, const double* __restrict__ v, double alpha,
                                double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double ur = alpha * u[r];
    for (int p = rp[r]; p < rp[r + 1]; ++p) out[p] += ur * v[col[p]];
}

void launch_pattern_outer(int n, const int* rp, const int* col, const double* u, const double* v, double alpha,
                          double* out, cudaStream_t st) {
    k_pattern_outer<<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, u, v, alpha, out);
    ++g_launches;
}

// Length class of a row: its length for rows of at most 16 entries, 17 for 17..64 entries, 18 for longer rows.
__device__ __forceinline__ int length_key(int len) { return len <= 16 ? len : (len <= 64 ? 17 : 18); }

// One CTA (256 threads) per row block: counting sort of the block's rows by length key, stable (rows of equal key
// keep their order), so the order -- and every sum formed in it -- is deterministic.
__global__ void __launch_bounds__(256) k_bin_rows(const int* __restrict__ rp, const int* __restrict__ lb_m0,
                                                  const int* __restrict__ lb_len, uint16_t* __restrict__ perm,
                                                  int* __restrict__ cls) {
    constexpr int NK = 19, NW = 8;
    __shared__ int cnt[NK], cur[NK], wc[NW][NK];
    const int L = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = lb_m0[L], len = lb_len[L];
    if (tid < NK) cnt[tid] = 0;
    __syncthreads();
    for (int k = tid; k < len; k += blockDim.x) atomicAdd(&cnt[length_key(rp[m0 + k + 1] - rp[m0 + k])], 1);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int b = 0; b < NK; ++b) {
            cur[b] = run;
            run += cnt[b];
        }
        cls[2 * L] = cur[17];
        cls[2 * L + 1] = cur[18];
    }
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < len; base += blockDim.x) {
        for (int q = tid; q < NW * NK; q += blockDim.x) wc[q / NK][q % NK] = 0;
        __syncthreads();
        const int k = base + tid;
        const bool ok = k < len;
        const int key = ok ? length_key(rp[m0 + k + 1] - rp[m0 + k]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (ok && lane == __ffs(peers) - 1) wc[warp][key] = __popc(peers);
        __syncthreads();
        if (ok) {
            int pos = cur[key] + __popc(peers & lt);
            for (int w = 0; w < warp; ++w) pos += wc[w][key];
            perm[m0 + pos] = (uint16_t)k;
        }
        __syncthreads();
        if (tid < NK) {
            int tot = 0;
            for (int w = 0; w < NW; ++w) tot += wc[w][tid];
            cur[tid] += tot;
        }
        __syncthreads();
    }
}

void launch_bin_rows(int nl, const int* rp, const int* lb_m0, const int* lb_len, uint16_t* perm, int* cls,
                     cudaStream_t st) {
    k_bin_rows<<<nl, 256, 0, st>>>(rp, lb_m0, lb_len, perm, cls);
    ++g_launches;
}

// ---- the length-binned SpMV's copy of a matrix: each row block's rows stored in their processing order ----
// Row i of block L's length order (local row perm[m0 + i]) is stored at brp[m0 + i] .. brp[m0 + i + 1] of bcol/bval,
// so the rows a warp processes together are neighbours in memory and every sector it loads is used while it is in L1
// (in CSR order the short rows of a warp lie among rows processed at other times, which share their sectors).

__global__ void k_bcopy_len(const int* __restrict__ rp, const int* __restrict__ lb_m0, const int* __restrict__ lb_len,
                            const uint16_t* __restrict__ perm, int* __restrict__ lens) {
    const int L = blockIdx.x;
    const int m0 = lb_m0[L], len = lb_len[L];
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int k = m0 + perm[m0 + i];
        lens[m0 + i] = rp[k + 1] - rp[k];
    }
}

// One warp per row: the row's entries copied in order (columns only when bcol is not null).
__global__ void k_bcopy_fill(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                             const int* __restrict__ lb_m0, const int* __restrict__ lb_len,
                             const uint16_t* __restrict__ perm, const int* __restrict__ brp, int* __restrict__ bcol,
                             double* __restrict__ bval) {
    const int L = blockIdx.x;
    const int m0 = lb_m0[L], len = lb_len[L];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < len; i += nw) {
        const int k = m0 + perm[m0 + i];
        const int a = rp[k], e = rp[k + 1], d = brp[m0 + i];
        for (int p = a + lane; p < e; p += 32) {
            if (bcol) bcol[d + (p - a)] = col[p];
            bval[d + (p - a)] = val[p];
        }
    }
}

void launch_bcopy_build(int n, int nl, const int* rp, const int* lb_m0, const int* lb_len, const uint16_t* perm,
                        int* lens, int* brp, cudaStream_t st) {
    k_bcopy_len<<<nl, 256, 0, st>>>(rp, lb_m0, lb_len, perm, lens);
    k_scan_plain<<<1, 1024, 0, st>>>(lens, brp, n);
    g_launches += 2;
}

void launch_bcopy_fill(int nl, const int* rp, const int* col, const double* val, const int* lb_m0,
                       const int* lb_len, const uint16_t* perm, const int* brp, int* bcol, double* bval,
                       cudaStream_t st) {
    k_bcopy_fill<<<nl, 256, 0, st>>>(rp, col, val, lb_m0, lb_len, perm, brp, bcol, bval);
    ++g_launches;
}

// ---- SELL-32 copy of a matrix with short rows ----
// Slice s holds rows moff[q] + 32 c .. of system q (c = s - sl0[q]); entry e of the slice's lane l sits at
// (off[s] + e) * 32 + l, so the 32 lanes of a warp read entry e of their rows with one coalesced load.  A slice is
// as wide as its longest row; a lane past its row's end (or past the system's last row) holds column 0, value 0,
// and its length says so.

__device__ __forceinline__ int sell_system(const int* __restrict__ sl0, int nsys, int64_t s) {
    int lo = 0, hi = nsys - 1;  // the last q with sl0[q] <= s
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sl0[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One warp per slice: row lengths and the slice width.
__global__ void k_sell_len(int ns, const int* __restrict__ sl0, int nsys, const int* __restrict__ moff,
                           const int* __restrict__ rp, uint8_t* __restrict__ len, int* __restrict__ wid) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = w0; s < ns; s += nwarps) {
        const int q = sell_system(sl0, nsys, s);
        const int r = moff[q] + 32 * (int)(s - sl0[q]) + lane;
        const int l = (r < moff[q + 1]) ? rp[r + 1] - rp[r] : 0;
        len[s * 32 + lane] = (uint8_t)l;
        const int w = (int)__reduce_max_sync(0xffffffffu, (unsigned)l);
        if (lane == 0) wid[s] = w;
    }
}

// One warp per slice: columns and values in slice order (entry order within each row).
__global__ void k_sell_fill(int ns, const int* __restrict__ sl0, int nsys, const int* __restrict__ moff,
                            const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                            const int* __restrict__ off, const uint8_t* __restrict__ len, int* __restrict__ scol,
                            double* __restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = w0; s < ns; s += nwarps) {
        const int q = sell_system(sl0, nsys, s);
        const int r = moff[q] + 32 * (int)(s - sl0[q]) + lane;
        const int l = len[s * 32 + lane];
        const int a = (l > 0) ? rp[r] : 0;
        const int64_t base = (int64_t)off[s] * 32 + lane;
        const int w = off[s + 1] - off[s];
        for (int e = 0; e < w; ++e) {
            if (scol) scol[base + (int64_t)e * 32] = (e < l) ? col[a + e] : 0;
            sval[base + (int64_t)e * 32] = (e < l) ? val[a + e] : 0.0;
        }
    }
}

static int sell_grid(int ns) { return (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)ns + 7) / 8, 152 * 64)); }

void launch_sell_build(int ns, const int* sl0, int nsys, const int* moff, const int* rp, uint8_t* len, int* wid,
                       int* off, cudaStream_t st) {
    k_sell_len<<<sell_grid(ns), 256, 0, st>>>(ns, sl0, nsys, moff, rp, len, wid);
    k_scan_plain<<<1, 1024, 0, st>>>(wid, off, ns);
    g_launches += 2;
}

void launch_sell_fill(int ns, const int* sl0, int nsys, const int* moff, const int* rp, const int* col,
                      const double* val, const int* off, const uint8_t* len, int* scol, double* sval,
                      cudaStream_t st) {
    k_sell_fill<<<sell_grid(ns), 256, 0, st>>>(ns, sl0, nsys, moff, rp, col, val, off, len, scol, sval);
    ++g_launches;
}

}  // namespace sfg
