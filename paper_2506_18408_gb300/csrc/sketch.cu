// Sparse-sign subspace embedding S (Eq. 1; Clarkson-Woodruff when zeta = 1, Section 4.1) on the device.
//
// S is never stored densely.  Each system's pattern is drawn once per sketch size from SplitMix64 (counter form, see
// sketch_column in common.cuh) and regrouped into *gather lists*: for each row block of the system (the blocks the
// fused inner kernel uses) and each sketch row r, the list of (local offset, sign) of the columns j in the block
// with S_rj != 0.  A kernel that holds the block of a vector in shared memory then forms its partial S x by summing
// each sketch row's list in a fixed order -- deterministic, no atomics on floating-point data.
//
// Layout: the sketch rows of a block form groups of 32 (group g: rows 32g .. 32g + 31, summed by the 32 lanes of one
// warp in lockstep).  A group's lists are stored interleaved in 16-byte units of 8 entries -- unit u of lane l at
// unit index gseg[k*ng + g] + 32u + l -- so that each load of a warp reads 512 contiguous bytes; every list of the
// group is padded to the group's longest (E units), with entries that point at the block's zero slot.
#include "kernels.h"

#include <algorithm>
#include <climits>
#include <mutex>
#include <unordered_map>

namespace sfg {

thread_local int64_t g_launches = 0;

void set_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(func);
    if (it != done.end() && it->second >= bytes) return;
    if (bytes > 48 * 1024) cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done[func] = bytes;
}

// Pattern: rows[j*zeta + l], neg[j*zeta + l] (1 = negative sign).  kind 1 = identity (zeta = 1, row = j).
__global__ void k_sketch_pattern(int n, int s, int zeta, int kind, uint64_t seed, int* __restrict__ rows,
                                 int8_t* __restrict__ neg) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (kind == 1) {
        rows[j] = (int)j;
        neg[j] = 0;
        return;
    }
    int r[kMaxZeta], ng[kMaxZeta];
    sketch_column(seed, j, zeta, s, r, ng);
    for (int l = 0; l < zeta; ++l) {
        rows[j * zeta + l] = r[l];
        neg[j * zeta + l] = (int8_t)ng[l];
    }
}

void launch_sketch_pattern(int n, int s, int zeta, int kind, uint64_t seed, int* rows, int8_t* neg,
                           cudaStream_t st) {
    k_sketch_pattern<<<(n + 255) / 256, 256, 0, st>>>(n, s, zeta, kind, seed, rows, neg);
    ++g_launches;
}

// counts[k*s + r] = number of nonzeros of sketch row r among the columns of block k (Bq columns per block)
__global__ void k_seg_count(int n, int s, int zeta, int Bq, const int* __restrict__ rows, int* __restrict__ counts) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int k = (int)(j / Bq);
    for (int l = 0; l < zeta; ++l) atomicAdd(counts + (int64_t)k * s + rows[j * zeta + l], 1);
}

// seg[0..len] = base + exclusive prefix sum of counts[0..len) (single block).
__global__ void k_scan_single(const int* __restrict__ counts, int* __restrict__ seg, int len, int base) {
    __shared__ int sums[1024];
    const int tid = threadIdx.x, T = blockDim.x;
    const int chunk = (len + T - 1) / T;
    const int a = min(len, tid * chunk), bnd = min(len, a + chunk);
    int local = 0;
    for (int i = a; i < bnd; ++i) local += counts[i];
    sums[tid] = local;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {  // Hillis-Steele inclusive scan of the per-thread totals
        int v = (tid >= off) ? sums[tid - off] : 0;
        __syncthreads();
        sums[tid] += v;
        __syncthreads();
    }
    int run = base + sums[tid] - local;
    for (int i = a; i < bnd; ++i) {
        seg[i] = run;
        run += counts[i];
    }
    if (tid == T - 1) seg[len] = base + sums[T - 1];
}

// units[k*ng + g] = 32 * E(k, g): the 16-byte units of group g of block k, E the group's longest list in units of
// 8 entries (counts[k*s + r]: the list lengths).
__global__ void k_group_units(int nl, int s, const int* __restrict__ counts, int* __restrict__ units) {
    const int ng = (s + 31) / 32;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nl * ng) return;
    const int k = (int)(t / ng), g = (int)(t % ng);
    int e = 0;
    for (int r = 32 * g; r < min(s, 32 * g + 32); ++r) e = max(e, (counts[(int64_t)k * s + r] + 7) >> 3);
    units[t] = 32 * e;
}

__global__ void k_fill_u16(int64_t cnt, uint16_t v, uint16_t* __restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = v;
}

// Fill the gather lists of block k (one warp per block; gseg: the block's group starts in units).  Entries of a list
// appear in the order (column chunk of 32, slot l, lane), which is fixed, so the sums formed from them are
// reproducible.
__global__ void k_seg_fill(int n, int s, int zeta, int Bq, const int* __restrict__ rows,
                           const int8_t* __restrict__ neg, const int* __restrict__ gseg,
                           uint16_t* __restrict__ ent) {
    const int ng = (s + 31) / 32;
    extern __shared__ int cursor[];
    const int k = blockIdx.x, lane = threadIdx.x;
    for (int r = lane; r < s; r += 32) cursor[r] = 0;
    __syncwarp();
    const int c0 = k * Bq, c1 = min(n, c0 + Bq);
    const unsigned lt = (1u << lane) - 1u;
    for (int base = c0; base < c1; base += 32) {
        const int j = base + lane;
        const bool ok = j < c1;
        for (int l = 0; l < zeta; ++l) {
            const int r = ok ? rows[(int64_t)j * zeta + l] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, r);
            if (ok) {
                const int e = cursor[r] + __popc(peers & lt);  // entry e of the list of row r
                const int64_t unit = (int64_t)gseg[(int64_t)k * ng + (r >> 5)] + 32 * (e >> 3) + (r & 31);
                ent[unit * 8 + (e & 7)] = (uint16_t)((j - c0) | (neg[(int64_t)j * zeta + l] ? 0x8000 : 0));
            }
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) cursor[r] += __popc(peers);
            __syncwarp();
        }
    }
}

// Reorders the entries within each gather list for the shared-memory banks.  The lanes of a warp sum the lists of
// their group in lockstep (entry e of every list at step e), and two lanes that share one shared-memory wavefront
// and read the same bank at a step serialise: G = 16 lanes (a half-warp) for the 8-byte words of the FP64
// fixed-point image, 32 for FP32 data; the bank of an entry is its offset mod G.  Each CTA takes the G lists of one
// half-group or group (G aligned) of one row block, all E * 8 entries long (padding included): they are bucketed by
// residue (stably, in shared memory), then step by step the lanes, in an order rotating with the step, each take the
// next entry of the residue that is least used at this step so far (ties: the lane's fullest bucket, then the lowest
// residue; bucket sizes compared up to 4095), each choice one warp-wide min-reduction over the residues.  Only the order within a list changes, and it is a fixed function of the list contents, so the sums stay
// reproducible (the FP64 ones are exact in any order).
template <int G>
__global__ void k_seg_schedule(int nl, int s, const int* __restrict__ gseg, uint16_t* __restrict__ ent) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int cnt[G * G], pos[G * G], cur[G * G], outp[G];
    uint16_t* buf = reinterpret_cast<uint16_t*>(smem_raw);
    const int ng = (s + 31) / 32;
    const int l = threadIdx.x;
    const int r0 = blockIdx.x * G, nr = min(G, s - r0);
    const int g = r0 >> 5, lo = r0 & 31;
    // position (in entries) of entry e of lane q of this group of lanes
    auto at = [&](int64_t gstart, int q, int e) -> int64_t { return (gstart + 32 * (e >> 3) + lo + q) * 8 + (e & 7); };
    for (int k = blockIdx.y; k < nl; k += gridDim.y) {
        const int64_t gstart = gseg[(int64_t)k * ng + g];
        const int L = 8 * ((gseg[(int64_t)k * ng + g + 1] - (int)gstart) / 32);  // entries per list
        for (int i = l; i < G * G; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        if (l < nr) {
            const int a = l * L;  // the lane's region of buf
            outp[l] = 0;
            for (int e = 0; e < L; ++e) ++cnt[l * G + (ent[at(gstart, l, e)] & 0x7fff) % G];
            int run = a;
            for (int r = 0; r < G; ++r) {
                pos[l * G + r] = run;
                cur[l * G + r] = run;
                run += cnt[l * G + r];
            }
            for (int e = 0; e < L; ++e) {
                const uint16_t v = ent[at(gstart, l, e)];
                buf[cur[l * G + (v & 0x7fff) % G]++] = v;
            }
        }
        __syncthreads();
        // the greedy, one lane per residue: for each list in turn the warp picks the residue with the smallest key
        // (uses at this step, then the list's fewer remaining entries of that residue, then the residue) with one
        // min-reduction; lane `pick` counts the use
        const bool own = l < G;  // this lane owns residue l
        for (int step = 0; step < L; ++step) {
            int used = 0;
            for (int q = 0; q < nr; ++q) {
                const int li = (step + q) % nr;
                const int c = own ? cnt[li * G + l] : 0;
                const unsigned key = (c > 0) ? ((unsigned)used << 20) | ((unsigned)(0xFFF - min(c, 0xFFF)) << 5) | (unsigned)l
                                             : 0xFFFFFFFFu;
                const unsigned best = __reduce_min_sync(0xffffffffu, key);
                const int pick = (int)(best & 31u);
                if (l == pick) {
                    ++used;
                    --cnt[li * G + pick];
                    ent[at(gstart, li, outp[li]++)] = buf[pos[li * G + pick]++];
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

void launch_sketch_schedule(int nl, int s, int word, int max_group, const int* gseg, uint16_t* ent, cudaStream_t st) {
    const size_t sm = ((size_t)max_group * sizeof(uint16_t) + 15) & ~(size_t)15;
    if (sm > 160 * 1024) return;  // very few sketch rows per block: the lists keep their fill order
    if (word == 8) {
        set_smem((const void*)k_seg_schedule<16>, sm);
        k_seg_schedule<16><<<dim3((s + 15) / 16, std::min(nl, 65535)), 32, sm, st>>>(nl, s, gseg, ent);
    } else {
        set_smem((const void*)k_seg_schedule<32>, sm);
        k_seg_schedule<32><<<dim3((s + 31) / 32, std::min(nl, 65535)), 32, sm, st>>>(nl, s, gseg, ent);
    }
    ++g_launches;
}

void launch_group_units(int nl, int s, const int* counts, int* units, cudaStream_t st) {
    const int64_t t = (int64_t)nl * ((s + 31) / 32);
    k_group_units<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(nl, s, counts, units);
    ++g_launches;
}

void launch_sketch_count(int n, int s, int zeta, int Bq, const int* rows, int* counts, cudaStream_t st) {
    k_seg_count<<<(n + 255) / 256, 256, 0, st>>>(n, s, zeta, Bq, rows, counts);
    ++g_launches;
}

void launch_list_scan(const int* counts, int* seg, int len, cudaStream_t st) {
    k_scan_single<<<1, 1024, 0, st>>>(counts, seg, len, 0);
    ++g_launches;
}

void launch_sketch_fill(int n, int s, int zeta, int Bq, const int* rows, const int8_t* neg, const int* gseg,
                        uint16_t* ent, cudaStream_t st) {
    const int nl = (n + Bq - 1) / Bq;
    k_seg_fill<<<nl, 32, s * sizeof(int), st>>>(n, s, zeta, Bq, rows, neg, gseg, ent);
    ++g_launches;
}

void launch_fill_u16(int64_t cnt, uint16_t v, uint16_t* out, cudaStream_t st) {
    k_fill_u16<<<(int)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, st>>>(cnt, v, out);
    ++g_launches;
}

// Per-block partial sketch of xs = scale_p * x; optionally stores (VT)xs into dst.  The value fed to the sketch is
// the stored (rounded) one, so S is applied to exactly the vector kept in the basis.  One thread per sketch row
// walks its gather list; FP64 data are summed exactly in 64-bit fixed point, FP32 data in list order.
template <typename VT, typename AT>
__global__ void __launch_bounds__(512) k_sketch_partials(const Plan P, const double* __restrict__ x,
                                                         const double* __restrict__ xscale, int xstride,
                                                         VT* __restrict__ dst, AT* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AT* xb = reinterpret_cast<AT*>(smem_raw);
    __shared__ int emax_sh[32];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    if (P.pflag[bi.prob] & 1) return;
    const int s = P.s, Bn = P.Bn;
    const double sc = xscale ? xscale[(int64_t)bi.prob * xstride] : 1.0;
    int emax = 1;
    for (int r = threadIdx.x; r <= Bn; r += blockDim.x) {
        AT v = AT(0);
        if (r < bi.len) {
            v = (AT)(sc * x[bi.v0 + r]);
            if (dst) {
                store_as(dst + bi.v0 + r, v);
                v = stored_value(v, dst);
            }
        }
        xb[r] = v;
        emax = max(emax, exp_of(v));
    }
    const int ng = (s + 31) / 32;
    const int* sg = P.seg + (int64_t)bi.list * ng;  // the block's group starts (units)
    if constexpr (sizeof(AT) == 8) {
        emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
        if ((threadIdx.x & 31) == 0) emax_sh[threadIdx.x >> 5] = emax;
        __syncthreads();
        int Eb = 1;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) Eb = max(Eb, emax_sh[q]);
        long long* qb = reinterpret_cast<long long*>(xb);
        for (int r = threadIdx.x; r <= Bn; r += blockDim.x) qb[r] = to_fixed((double)xb[r], Eb, P.sk_headroom);
        __syncthreads();
        const double unit = fixed_unit(0.0, Eb, P.sk_headroom);
        const bool bad = exp_nonfinite(0.0, Eb);
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            const int g = rr >> 5;
            const long long v = sum_group(P.ent, sg[g], (sg[g + 1] - sg[g]) >> 5, rr & 31, qb);
            part[(int64_t)b * s + rr] = bad ? (AT)NAN : (AT)((double)v * unit);
        }
    } else {
        __syncthreads();
        for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
            const int g = rr >> 5;
            part[(int64_t)b * s + rr] = sum_group(P.ent, sg[g], (sg[g + 1] - sg[g]) >> 5, rr & 31, xb);
        }
    }
}

void launch_sketch_partials(const Plan& p, const double* x, const double* xscale, int xstride, void* dst,
                            void* part) {
    const size_t sm = (size_t)(p.Bn + 1) * (p.prec == kFP64 ? 8 : 4);
    if (p.prec == kFP64) {
        set_smem((const void*)k_sketch_partials<double, double>, sm);
        k_sketch_partials<double, double><<<p.nblk, 512, sm, p.st>>>(p, x, xscale, xstride, (double*)dst,
                                                                    (double*)part);
    } else if (p.prec == kFP32) {
        set_smem((const void*)k_sketch_partials<float, float>, sm);
        k_sketch_partials<float, float><<<p.nblk, 512, sm, p.st>>>(p, x, xscale, xstride, (float*)dst,
                                                                  (float*)part);
    } else {
        set_smem((const void*)k_sketch_partials<__nv_bfloat16, float>, sm);
        k_sketch_partials<__nv_bfloat16, float><<<p.nblk, 512, sm, p.st>>>(p, x, xscale, xstride,
                                                                          (__nv_bfloat16*)dst, (float*)part);
    }
    ++g_launches;
}

// out[p*s + r] = sk_scale * sum over the blocks of problem p of part[b*s + r]: one warp per (p, r), lane l summing
// blocks b0 + l, b0 + l + 32, ... in order with all its loads issued first, then the warp's shuffle tree (a fixed
// order: reproducible).
template <typename AT>
__global__ void k_sketch_reduce(const Plan P, const AT* __restrict__ part, double* __restrict__ out,
                                double* __restrict__ out2) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int s = P.s;
    if (t >= (int64_t)P.P * s) return;  // warp-uniform
    const int p = (int)(t / s), r = (int)(t % s);
    if (P.pflag[p] & 1) return;
    const int b0 = P.prob_b0[p], b1 = P.prob_b0[p + 1];
    AT acc = AT(0);
    for (int q0 = b0 + lane; q0 < b1; q0 += 128) {
        AT v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (q0 + 32 * u < b1) ? part[(int64_t)(q0 + 32 * u) * s + r] : AT(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += v[u];
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        const double v = P.sk_scale * (double)acc;
        out[t] = v;
        if (out2) out2[t] = v;
    }
}

void launch_sketch_reduce(const Plan& p, const void* part, double* out, double* out2) {
    const int64_t warps = (int64_t)p.P * p.s;
    const int th = 256, gr = (int)((warps * 32 + th - 1) / th);
    if (p.prec == kFP64)
        k_sketch_reduce<double><<<gr, th, 0, p.st>>>(p, (const double*)part, out, out2);
    else
        k_sketch_reduce<float><<<gr, th, 0, p.st>>>(p, (const float*)part, out, out2);
    ++g_launches;
}

}  // namespace sfg
