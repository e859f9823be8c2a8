// One whole sketched-GMRES cycle (Section 3) per launch for problems of at most kPersistCluster row blocks: the
// persistent form of the per-step kernels in inner.cu, for systems small enough that launch latency, not memory
// traffic, bounds the per-step kernels.
//
// One cluster of kPersistCluster CTAs per problem; CTA q owns the problem's q-th row block (CTAs beyond the problem's
// blocks own none and only take part in the reductions).  Each inner step i runs, inside the kernel:
//   w' = A u_i with the window dots u_l^T w' and ||u_i||^2 on the CTA's rows, and the block's sketch partial S w'
//   -> cluster barrier -> every CTA sums the CTAs' partials in rank order through distributed shared memory
//   (identical values in every CTA, so every decision below is taken identically everywhere): sigma_i, the
//   truncated-Arnoldi coefficients, the CTA's rows of the sketched column S A b_i
//   -> u_{i+1} = 2^p (w' - sum_l sigma_l^2 (u_l^T w') u_l) on the CTA's rows
//   -> the Gram-Schmidt update of the sketched QR with one reorthogonalisation pass, distributed over the CTAs by
//   sketch rows (each CTA keeps its rows of Q and of the sketched residual in shared memory; partials
//   double-buffered by pass; ||p|| and p^T e exchanged together), the condition proxy (C2)
//   and C1; the sketched residual of the accepted column is exchanged with the next step's partials and rule C3 is
//   applied there (the next step's SpMV is then discarded, as the per-step kernels discard a step past the end).
// Four cluster barriers per step; the barriers after the update of u_{i+1} also order it before the next SpMV.
// After the last step rank 0 solves R_k y = d, and every CTA forms its rows of z = B_k y.  The arithmetic of each
// step is that of k_inner_spmv / k_inner_axpy / k_inner_qr (same sums, block partials in the same order; the block
// reductions run warp by warp).  Every wait is a hardware cluster barrier reached by all CTAs of the cluster the same
// number of times: the loop exits on values every CTA holds identically.
#include "kernels.h"
#include "spmv.cuh"

#include <algorithm>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace sfg {

// Loads that bypass L1 and the read-only path: the data were written by other CTAs of this launch.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const __nv_bfloat16* p) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float((unsigned)b << 16);
}

// CNT entries of one row chunk with coherent gathers (the vector was written by other CTAs of this launch).
template <int CNT, typename MT, typename XT, typename AT>
__device__ __forceinline__ void row_chunk_cg(const int* __restrict__ col, const MT* __restrict__ val,
                                             const XT* x, int a, int len, int pk, AT& sum) {
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
        if (pk + q < len) sum += v[q] * (AT)ld_cg(x + c[q]);
}

// Per-CTA scratch of the persistent cycle (static part; the row block of w' and the sketch partial are dynamic).
template <typename AT>
struct PersistSm {
    double part[kMaxTrunc + 1];  // this CTA's ||u_i||^2 and window dots
    AT red[kMaxTrunc + 1][16];
    int emax[16];
    double coef[kMaxTrunc];
    double scal[4];              // this CTA's QR partials: ||p||^2, p^T e, ||e||^2 after the update
    double tot[kMaxTrunc + 1];   // cluster totals; tot[kMaxTrunc] = ||e||^2 of the last accepted column
    double red64[32];
};

template <int NW, typename MT, typename VT, typename AT>
__device__ __forceinline__ void persist_spmv_dots(const Plan& P, const MT* __restrict__ val, int i, int v0, int len,
                                                  int cs, AT* __restrict__ wblk, AT (&acc)[kMaxTrunc], AT& nrm,
                                                  int& emax) {
    const int lane = threadIdx.x & 31, N = P.N;
    const VT* Ub = (const VT*)P.U;
    const VT* xs = Ub + (int64_t)i * N + cs;
    const int* rpm = P.rp + (v0 - cs);
    const int lo = i - NW + 1;
    for (int kw = threadIdx.x & ~31; kw < len; kw += blockDim.x) {  // warp-uniform loop over the block's rows
        const int k = kw + lane;
        const bool ok = k < len;
        const int r = v0 + k;
        int a = 0, rl = 0;
        if (ok) {
            a = __ldg(rpm + k);
            rl = __ldg(rpm + k + 1) - a;
        }
        AT uw[NW > 0 ? NW : 1];
#pragma unroll
        for (int q = 0; q < NW; ++q) uw[q] = ok ? ld_plain(Ub + (int64_t)(lo + q) * N + r) : AT(0);
        AT ui;
        if constexpr (NW > 0) ui = uw[NW - 1];
        else ui = ok ? ld_plain(Ub + (int64_t)i * N + r) : AT(0);
        const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)rl);
        AT sum = AT(0);
        for (int pk = 0; pk < maxlen; pk += 4) {
            switch (min(maxlen - pk, 4)) {
                case 1: row_chunk_cg<1>(P.col, val, xs, a, rl, pk, sum); break;
                case 2: row_chunk_cg<2>(P.col, val, xs, a, rl, pk, sum); break;
                case 3: row_chunk_cg<3>(P.col, val, xs, a, rl, pk, sum); break;
                default: row_chunk_cg<4>(P.col, val, xs, a, rl, pk, sum); break;
            }
        }
        if (ok) wblk[k] = sum;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc[q] += uw[q] * sum;
        nrm += ui * ui;
        emax = max(emax, exp_of(sum));
    }
}

template <int NW, typename VT, typename AT>
__device__ __forceinline__ void persist_axpy(const Plan& P, int i, int v0, int len, const AT* __restrict__ wblk,
                                             const double* __restrict__ coef, double sig_i) {
    const int N = P.N, lo = i - NW + 1;
    VT* Ub = (VT*)P.U;
    int p2;
    frexp(sig_i, &p2);
    p2 -= 1;
    const AT sc2 = (AT)ldexp(1.0, p2);
    AT cf[NW > 0 ? NW : 1];
#pragma unroll
    for (int q = 0; q < NW; ++q) cf[q] = (AT)coef[q];
    VT* un = Ub + (int64_t)(i + 1) * N;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const int r = v0 + k;
        AT u = wblk[k];
#pragma unroll
        for (int q = 0; q < NW; ++q) u -= cf[q] * ld_plain(Ub + (int64_t)(lo + q) * N + r);
        if constexpr (sizeof(AT) == 8) u = mul_pow2((double)u, p2);
        else u = u * sc2;
        store_as(un + r, u);
    }
}

// Sum over the cluster's ranks, in rank order, of the double at offset `off` of every CTA's shared-memory array
// `base` (all loads issued before the adds).
__device__ __forceinline__ double rank_sum(cg::cluster_group& cl, double* base, int off, int nq) {
    double v[kPersistCluster];
#pragma unroll
    for (int r2 = 0; r2 < kPersistCluster; ++r2) v[r2] = (r2 < nq) ? cl.map_shared_rank(base, r2)[off] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int r2 = 0; r2 < kPersistCluster; ++r2) acc += v[r2];
    return acc;
}

template <typename MT, typename VT, typename AT>
__global__ void __launch_bounds__(512, 1) k_cycle_persistent(const Plan P, double* __restrict__ z) {
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank(), nq = (int)cl.num_blocks();
    const int prob = blockIdx.x / nq;
    const int s = P.s, m = P.m, t = P.t, N = P.N, Bn = P.Bn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (P.pflag[prob] & 1) return;  // the whole cluster returns (the flag is the same for every CTA)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // dynamic: wblk [Bn + 1] (AT, the block of w'), qfix [Bn + 1] (its fixed-point image, FP64), cps [s] (this
    // CTA's sketch partial), pv [nrmax] (QR working rows), apart [2][m] (CGS partials, one buffer per pass),
    // av [m], sig [m + 1], ycoef [m] (doubles)
    const int nrmax = (s + nq - 1) / nq;
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    long long* qfix = reinterpret_cast<long long*>(smem_raw + (((size_t)(Bn + 1) * sizeof(AT) + 15) & ~(size_t)15));
    double* cps = reinterpret_cast<double*>(qfix + (sizeof(AT) == 8 ? (((Bn + 1) + 1) & ~1) : 0));
    double* pv = cps + s;
    double* apart = pv + nrmax;
    double* av = apart + 2 * m;
    double* sig = av + m;
    double* ycoef = sig + m + 1;
    double* es = ycoef + m;        // this CTA's rows of the running sketched residual e
    double* Qs = es + nrmax;       // this CTA's rows of Q: Qs[l * nrmax + r]
    __shared__ PersistSm<AT> S;

    const int b0 = P.prob_b0[prob], nb = P.prob_b0[prob + 1] - b0;
    const bool own = q < nb;
    BlockInfo bi = {0, 0, 0, 0, prob};
    if (own) bi = block_info(P, b0 + q);
    const MT* val = (P.prec == kFP64) ? (const MT*)P.val : (const MT*)P.val32;
    const int rlo = (int)((int64_t)s * q / nq), rhi = (int)((int64_t)s * (q + 1) / nq), nr = rhi - rlo;
    double* __restrict__ R = P.R + (int64_t)prob * m * m;
    double* __restrict__ d = P.d + (int64_t)prob * m;
    const double* __restrict__ e0 = P.e + (int64_t)prob * s;  // S v (set at the cycle start)
    double* __restrict__ rho = P.rho + (int64_t)prob * m;
    CycleState* cyc = P.cyc + prob;
    const double c3_scale = cyc->c3_scale, c3_tol = cyc->c3_tol, thr = cyc->cond_thr;
    const int c3_on = cyc->c3_on;
    const int* sg = P.seg + (int64_t)bi.list * s;
    for (int l = threadIdx.x; l <= m; l += blockDim.x) sig[l] = (l == 0) ? 1.0 : 0.0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) es[r] = e0[rlo + r];
    double dmax = 0.0, dmin = INFINITY;
    int k_acc = 0, reason = 0;
    bool rho_pending = false;  // the last accepted column's ||e||^2 partials await the next exchange
    cl.sync();
    for (int i = 0; i < m; ++i) {
        const int NWi = (t > 0) ? min(t, i + 1) : 0;
        const int lo = i - NWi + 1;
        // ---- w' = A u_i, window dots, ||u_i||^2, sketch partial (own block) ----
        AT acc[kMaxTrunc];
#pragma unroll
        for (int qq = 0; qq < kMaxTrunc; ++qq) acc[qq] = AT(0);
        AT nrm = AT(0);
        int emax = 1;
        if (own) {
            switch (NWi) {
                case 0: persist_spmv_dots<0, MT, VT, AT>(P, val, i, bi.v0, bi.len, bi.cs, wblk, acc, nrm, emax); break;
                case 1: persist_spmv_dots<1, MT, VT, AT>(P, val, i, bi.v0, bi.len, bi.cs, wblk, acc, nrm, emax); break;
                case 2: persist_spmv_dots<2, MT, VT, AT>(P, val, i, bi.v0, bi.len, bi.cs, wblk, acc, nrm, emax); break;
                case 3: persist_spmv_dots<3, MT, VT, AT>(P, val, i, bi.v0, bi.len, bi.cs, wblk, acc, nrm, emax); break;
                default: persist_spmv_dots<4, MT, VT, AT>(P, val, i, bi.v0, bi.len, bi.cs, wblk, acc, nrm, emax); break;
            }
        }
        if (threadIdx.x == 0) wblk[Bn] = AT(0);
        {
            const AT v = warp_sum(nrm);
            if (lane == 0) S.red[0][warp] = v;
            for (int qq = 0; qq < NWi; ++qq) {
                const AT dd = warp_sum(acc[qq]);
                if (lane == 0) S.red[1 + qq][warp] = dd;
            }
            emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
            if (lane == 0) S.emax[warp] = emax;
        }
        __syncthreads();
        if (threadIdx.x <= NWi) {
            AT tt = AT(0);
            for (int w = 0; w < nw; ++w) tt += S.red[threadIdx.x][w];
            S.part[threadIdx.x] = own ? (double)tt : 0.0;
        }
        if (own) {
            if constexpr (sizeof(AT) == 8) {
                // exact fixed-point sketch sums over the block's image (every thread converts its rows first)
                int Eb = 1;
                for (int w = 0; w < nw; ++w) Eb = max(Eb, S.emax[w]);
                const int H = P.sk_headroom;
                for (int r = threadIdx.x; r <= Bn; r += blockDim.x)
                    qfix[r] = (r < bi.len) ? to_fixed((double)wblk[r], Eb, H) : 0;
                __syncthreads();
                const double unit = fixed_unit(0.0, Eb, H);
                const bool badx = exp_nonfinite(0.0, Eb);
                for (int rr = threadIdx.x; rr < s; rr += blockDim.x) {
                    const long long v = sum_list(P.ent, sg[rr], sg[rr + 1], qfix);
                    cps[rr] = badx ? NAN : (double)v * unit;
                }
            } else {
                for (int rr = threadIdx.x; rr < s; rr += blockDim.x)
                    cps[rr] = (double)sum_list(P.ent, sg[rr], sg[rr + 1], wblk);
            }
        } else {
            for (int rr = threadIdx.x; rr < s; rr += blockDim.x) cps[rr] = 0.0;
        }
        cl.sync();  // [1] this step's partials, and the previous accepted column's ||e||^2 partials
        // ---- totals in rank order (the same values in every CTA) ----
        if (threadIdx.x <= NWi) S.tot[threadIdx.x] = rank_sum(cl, S.part, threadIdx.x, nq);
        if (threadIdx.x == 32) S.tot[kMaxTrunc] = rank_sum(cl, S.scal, 2, nq);
        __syncthreads();
        if (rho_pending) {  // rule C3 for the column accepted at step i - 1
            const double rh = sqrt(S.tot[kMaxTrunc]);
            if (q == 0 && threadIdx.x == 0) rho[i - 1] = rh;
            rho_pending = false;
            if (c3_on && c3_scale * rh <= c3_tol) {
                reason = 3;
                break;
            }
        }
        double sig_i = sig[0];
        bool bad = false;
        int why = 4;
        if (i > 0) {
            const double a2 = S.tot[0];
            bad = !(a2 > 0.0) || !isfinite(a2);
            why = (a2 == 0.0) ? 4 : 6;
            sig_i = 1.0 / sqrt(a2);
        }
        if (bad) {  // u_i has zero (or non-finite) norm: the cycle keeps k = i columns
            reason = why;
            break;
        }
        if (threadIdx.x == 0) {
            sig[i] = sig_i;
            for (int qq = 0; qq < NWi; ++qq) {
                const int l = lo + qq;
                const double sl = (l == i) ? sig_i : sig[l];
                S.coef[qq] = sl * sl * S.tot[1 + qq];
            }
        }
        // ---- this CTA's rows of the sketched column S A b_i ----
        const double csc = P.sk_scale * sig_i;
        for (int r = threadIdx.x; r < nr; r += blockDim.x) pv[r] = csc * rank_sum(cl, cps, rlo + r, nq);
        __syncthreads();
        // ---- next stored basis vector on the CTA's rows (complete on every CTA before barrier [2]) ----
        if (own && i + 1 < m) {
            switch (NWi) {
                case 0: persist_axpy<0, VT, AT>(P, i, bi.v0, bi.len, wblk, S.coef, sig_i); break;
                case 1: persist_axpy<1, VT, AT>(P, i, bi.v0, bi.len, wblk, S.coef, sig_i); break;
                case 2: persist_axpy<2, VT, AT>(P, i, bi.v0, bi.len, wblk, S.coef, sig_i); break;
                case 3: persist_axpy<3, VT, AT>(P, i, bi.v0, bi.len, wblk, S.coef, sig_i); break;
                default: persist_axpy<4, VT, AT>(P, i, bi.v0, bi.len, wblk, S.coef, sig_i); break;
            }
        }
        // ---- sketched QR: Gram-Schmidt with one reorthogonalisation pass (partials double-buffered) ----
        for (int pass = 0; pass < 2; ++pass) {
            double* ap = apart + pass * m;
            for (int l = threadIdx.x; l < i; l += blockDim.x) {
                const double* ql = Qs + (int64_t)l * nrmax;
                double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
                int r = 0;
                for (; r + 4 <= nr; r += 4) {
                    c0 += ql[r] * pv[r];
                    c1 += ql[r + 1] * pv[r + 1];
                    c2 += ql[r + 2] * pv[r + 2];
                    c3 += ql[r + 3] * pv[r + 3];
                }
                for (; r < nr; ++r) c0 += ql[r] * pv[r];
                ap[l] = (c0 + c1) + (c2 + c3);
            }
            cl.sync();  // [2], [3]
            for (int l = threadIdx.x; l < i; l += blockDim.x) av[l] = rank_sum(cl, ap, l, nq);
            __syncthreads();
            for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                const double* qr = Qs + r;
                double v0 = pv[r], v1 = 0.0, v2 = 0.0, v3 = 0.0;
                int l = 0;
                for (; l + 4 <= i; l += 4) {
                    v0 -= av[l] * qr[l * nrmax];
                    v1 -= av[l + 1] * qr[(l + 1) * nrmax];
                    v2 -= av[l + 2] * qr[(l + 2) * nrmax];
                    v3 -= av[l + 3] * qr[(l + 3) * nrmax];
                }
                for (; l < i; ++l) v0 -= av[l] * qr[l * nrmax];
                pv[r] = (v0 + v1) + (v2 + v3);
            }
            if (q == 0)
                for (int l = threadIdx.x; l < i; l += blockDim.x)
                    R[(int64_t)i * m + l] = (pass ? R[(int64_t)i * m + l] : 0.0) + av[l];
            __syncthreads();
        }
        // ---- r_ii = ||p|| and p^T e in one exchange; q_i = p / r_ii, d_i = q_i^T e ----
        {
            double v2 = 0.0, pe = 0.0;
            for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                v2 += pv[r] * pv[r];
                pe += pv[r] * es[r];
            }
            v2 = warp_sum(v2);
            pe = warp_sum(pe);
            if (lane == 0) {
                S.red64[warp] = v2;
                S.red64[16 + warp] = pe;
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                double tt = 0.0;
                for (int w = 0; w < nw; ++w) tt += S.red64[16 * threadIdx.x + w];
                S.scal[threadIdx.x] = tt;
            }
        }
        cl.sync();  // [4]
        if (threadIdx.x < 2) S.tot[threadIdx.x] = rank_sum(cl, S.scal, threadIdx.x, nq);
        __syncthreads();
        const double rii = sqrt(S.tot[0]);
        const double dmx = fmax(dmax, rii);
        const double dmn = (i == 0) ? rii : fmin(dmin, rii);
        const double kappa = (dmn > 0.0) ? dmx / dmn : INFINITY;
        if (!(kappa <= thr)) {  // C2 (also rii == 0 or NaN): drop column i, keep k = i
            reason = (i == 0) ? 5 : 2;
            break;
        }
        dmax = dmx;
        dmin = dmn;
        const double inv = 1.0 / rii;
        const double di = S.tot[1] * inv;
        double ee = 0.0;
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
            const double qv = pv[r] * inv;
            Qs[i * nrmax + r] = qv;
            const double ev = es[r] - di * qv;
            es[r] = ev;
            ee += ev * ev;
        }
        ee = warp_sum(ee);
        if (lane == 0) S.red64[warp] = ee;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tt = 0.0;
            for (int w = 0; w < nw; ++w) tt += S.red64[w];
            S.scal[2] = tt;  // exchanged at the next barrier [1] (or after the loop)
            if (q == 0) {
                R[(int64_t)i * m + i] = rii;
                d[i] = di;
            }
        }
        k_acc = i + 1;
        rho_pending = true;
        if (i + 1 == m) {  // C1
            reason = 1;
            break;
        }
    }
    // ---- y = R_k^{-1} d (rank 0, one warp), coef_l = y_l sigma_l; z = sum_l coef_l u_l on every CTA's rows ----
    const int k = k_acc;
    cl.sync();
    if (rho_pending && threadIdx.x == 0) {  // the last column's sketched residual (the cycle ended by C1)
        const double rh = sqrt(rank_sum(cl, S.scal, 2, nq));
        if (q == 0) rho[k - 1] = rh;
        if (c3_on && c3_scale * rh <= c3_tol) reason = 3;  // C3 is tested before C1, as the per-step kernels do
    }
    if (q == 0 && warp == 0) {
        for (int l = lane; l < k; l += 32) ycoef[l] = d[l];
        __syncwarp();
        for (int l = k - 1; l >= 0; --l) {
            const double yl = ycoef[l] / R[(int64_t)l * m + l];
            for (int qq = lane; qq < l; qq += 32) ycoef[qq] -= R[(int64_t)l * m + qq] * yl;
            __syncwarp();
            if (lane == 0) {
                ycoef[l] = yl;
                P.y[(int64_t)prob * m + l] = yl;
                P.coef[(int64_t)prob * m + l] = yl * sig[l];
            }
            __syncwarp();
        }
        for (int l = lane; l < k; l += 32) ycoef[l] *= sig[l];
    }
    cl.sync();
    if (q != 0)
        for (int l = threadIdx.x; l < k; l += blockDim.x) ycoef[l] = cl.map_shared_rank(ycoef, 0)[l];
    if (q == 0)
        for (int l = threadIdx.x; l <= m; l += blockDim.x) P.sigma[(int64_t)prob * (m + 1) + l] = sig[l];
    cl.sync();  // no CTA leaves or overwrites its shared memory while another may still read it
    if (own) {
        const VT* Ub = (const VT*)P.U;
        for (int kk = threadIdx.x; kk < bi.len; kk += blockDim.x) {
            const int64_t r = bi.v0 + kk;
            if constexpr (sizeof(VT) == 8) {
                double accz = 0.0;
                for (int l = 0; l < k; ++l) accz += ycoef[l] * (double)ld_plain(Ub + (int64_t)l * N + r);
                z[r] = accz;
            } else {
                float sh = 0.f, sl = 0.f;
                for (int l = 0; l < k; ++l) {
                    const float u = ld_plain(Ub + (int64_t)l * N + r);
                    const float ch = (float)ycoef[l];
                    const float cl2 = (float)(ycoef[l] - (double)ch);
                    const float pr = ch * u;
                    const float pe = fmaf(ch, u, -pr) + cl2 * u;
                    const float t1 = sh + pr;
                    const float bv = t1 - sh;
                    const float er = (sh - (t1 - bv)) + (pr - bv);
                    sh = t1;
                    sl += er + pe;
                }
                z[r] = (double)sh + (double)sl;
            }
        }
    }
    if (q == 0 && threadIdx.x == 0) {
        cyc->k = k;
        cyc->reason = reason;
        cyc->stopped = 1;
        cyc->dmax = dmax;
        cyc->dmin = dmin;
    }
}

size_t persistent_smem(const Plan& p, int nq) {
    const size_t at = (p.prec == kFP64) ? 8 : 4;
    const int nrmax = (p.s + nq - 1) / nq;
    const size_t fix = (p.prec == kFP64) ? (size_t)(((p.Bn + 1) + 1) & ~1) * 8 : 0;
    return (((size_t)(p.Bn + 1) * at + 15) & ~(size_t)15) + fix +
           (size_t)(p.s + nrmax + 3 * p.m + (p.m + 1) + p.m + nrmax + (size_t)p.m * nrmax) * sizeof(double);
}

cudaError_t launch_cycle_persistent(const Plan& p, int nq, double* z) {
    const size_t sm = persistent_smem(p, nq);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nq * p.P), 1, 1);
    cfg.blockDim = dim3(512, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = p.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nq;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++g_launches;
    if (p.prec == kFP64) {
        set_smem((const void*)k_cycle_persistent<double, double, double>, sm);
        return cudaLaunchKernelEx(&cfg, k_cycle_persistent<double, double, double>, p, z);
    }
    if (p.prec == kFP32) {
        set_smem((const void*)k_cycle_persistent<float, float, float>, sm);
        return cudaLaunchKernelEx(&cfg, k_cycle_persistent<float, float, float>, p, z);
    }
    set_smem((const void*)k_cycle_persistent<float, __nv_bfloat16, float>, sm);
    return cudaLaunchKernelEx(&cfg, k_cycle_persistent<float, __nv_bfloat16, float>, p, z);
}

}  // namespace sfg
