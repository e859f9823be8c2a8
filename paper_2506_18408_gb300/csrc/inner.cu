// One sketched-GMRES cycle on the device (Section 3; Eq. 3 with r0 = v_j and zero initial guess).
//
// Per inner step i (0-based; the paper's i+1):
//   k_inner_spmv  w = A b_i (b_i = sigma_i u_i), the truncated-Arnoldi dot products u_l^T w for the last t basis
//                 vectors (Section 4.1), and the per-block partial sketch of w -- all from one pass over A, with the
//                 row block of w held in shared memory for the sketch gather lists.
//   k_inner_axpy  reduces the dots (every CTA, same order) and its slice of the sketch partials into the column
//                 S A b_i, then u_{i+1} = w - sum_l h_l b_l and per-block partial ||u_{i+1}||^2.  The norm is reduced
//                 by the next step's k_inner_spmv, which folds 1/||u_{i+1}|| into its SpMV (deferred normalisation).
//   k_inner_qr    one CTA: Gram-Schmidt with one reorthogonalisation pass of S A b_i against Q (Section 3, C2), the
//                 condition proxy max|r_ll|/min|r_ll| (rule C2), the running sketched residual (rule C3) and C1.
// After the cycle: k_inner_finish solves R_k y = Q_k^T S v_j and forms z_j = B_k y_k in FP64.
#include "kernels.h"
#include "spmv.cuh"

#include <algorithm>

namespace sfg {

// ---------------------------------------------------------------------------------------------------------------
template <int V, int U, typename MT, typename VT, typename AT>
__global__ void __launch_bounds__(512, 2)
    k_inner_spmv(int n, int Bn, int nblk, int s, int t, int i, const int* __restrict__ rp,
                 const int* __restrict__ col, const MT* __restrict__ val, const VT* __restrict__ Ub,
                 AT* __restrict__ W, double* __restrict__ sigma, const AT* __restrict__ normpart,
                 AT* __restrict__ hpart, AT* __restrict__ cpart, const int* __restrict__ seg,
                 const uint16_t* __restrict__ ent, CycleState* __restrict__ cyc) {
    extern __shared__ unsigned char smem_raw[];
    AT* wblk = reinterpret_cast<AT*>(smem_raw);
    __shared__ AT red[32];
    __shared__ AT sig_sh;
    __shared__ int stop_sh;
    if (threadIdx.x == 0) stop_sh = cyc->stopped;
    __syncthreads();
    if (stop_sh) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    // sigma_i: 1/||u_i|| from the previous step's per-block partials (same fixed order in every CTA)
    if (warp == 0) {
        AT sig;
        if (i == 0) {
            sig = (AT)sigma[0];
        } else {
            AT acc = AT(0);
            for (int q = lane; q < nblk; q += 32) acc += normpart[q];
            acc = warp_sum(acc);
            sig = AT(1) / sqrt(acc);
            if (lane == 0) {
                const bool bad = !(acc > AT(0)) || !isfinite((double)acc);
                if (b == 0) sigma[i] = (double)sig;
                if (bad) {
                    if (b == 0) {
                        cyc->stopped = 1;  // eta == 0: invariant Krylov space (k stays i); NaN: stop too
                        cyc->reason = (acc == AT(0)) ? 4 : 6;
                    }
                    stop_sh = 1;
                }
            }
        }
        if (lane == 0) sig_sh = sig;
    }
    __syncthreads();
    if (stop_sh) return;
    const AT sig = sig_sh;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    const VT* x = Ub + (int64_t)i * n;
    spmv_rows_to_smem<V, U, MT, VT, AT>(rp, col, val, x, r0, r1, sig, wblk);
    __syncthreads();
    // w to global and the truncated-Arnoldi dots against u_lo..u_i
    const int lo = (t > 0) ? max(0, i - t + 1) : i + 1;
    const int nwin = i + 1 - lo;
    AT acc[kMaxTrunc];
#pragma unroll
    for (int q = 0; q < kMaxTrunc; ++q) acc[q] = AT(0);
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const AT w = wblk[r - r0];
        W[r] = w;
#pragma unroll
        for (int q = 0; q < kMaxTrunc; ++q)
            if (q < nwin) acc[q] += ld_plain(Ub + (int64_t)(lo + q) * n + r) * w;
    }
#pragma unroll
    for (int q = 0; q < kMaxTrunc; ++q) {
        if (q < nwin) {
            const AT v = block_sum(acc[q], red);
            if (threadIdx.x == 0) hpart[(int64_t)b * kMaxTrunc + q] = v;
        }
    }
    // partial sketch of w: one warp per sketch row, fixed order
    for (int rr = warp; rr < s; rr += nw) {
        const int a = seg[(int64_t)b * s + rr], e = seg[(int64_t)b * s + rr + 1];
        AT sacc = AT(0);
        for (int q = a + lane; q < e; q += 32) {
            const unsigned en = ent[q];
            const AT v = wblk[en & 0x7fffu];
            sacc += (en & 0x8000u) ? -v : v;
        }
        sacc = warp_sum(sacc);
        if (lane == 0) cpart[(int64_t)b * s + rr] = sacc;
    }
}

// ---------------------------------------------------------------------------------------------------------------
template <typename VT, typename AT>
__global__ void __launch_bounds__(512)
    k_inner_axpy(int n, int Bn, int nblk, int s, int t, int i, int last, double sk_scale, VT* __restrict__ Ub,
                 const AT* __restrict__ W, const double* __restrict__ sigma, AT* __restrict__ normpart,
                 const AT* __restrict__ hpart, const AT* __restrict__ cpart, double* __restrict__ C,
                 double* __restrict__ hco, CycleState* __restrict__ cyc) {
    __shared__ AT red[32];
    __shared__ AT coef_sh[kMaxTrunc];
    __shared__ int stop_sh;
    if (threadIdx.x == 0) stop_sh = cyc->stopped;
    __syncthreads();
    if (stop_sh) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x;
    const int lo = (t > 0) ? max(0, i - t + 1) : i + 1;
    const int nwin = i + 1 - lo;
    // h_l = sigma_l * (u_l^T w); the update coefficient of u_l is h_l * sigma_l
    if (warp < nwin) {
        AT acc = AT(0);
        for (int q = lane; q < nblk; q += 32) acc += hpart[(int64_t)q * kMaxTrunc + warp];
        acc = warp_sum(acc);
        if (lane == 0) {
            const AT sl = (AT)sigma[lo + warp];
            const AT h = sl * acc;
            coef_sh[warp] = h * sl;
            if (b == 0) hco[(int64_t)i * kMaxTrunc + warp] = (double)h;
        }
    }
    // this CTA's slice of the sketch column S A b_i
    for (int rr = b * blockDim.x + threadIdx.x; rr < s; rr += gridDim.x * blockDim.x) {
        AT acc = AT(0);
        for (int q = 0; q < nblk; ++q) acc += cpart[(int64_t)q * s + rr];
        C[(int64_t)i * s + rr] = sk_scale * (double)acc;
    }
    if (last) return;
    __syncthreads();
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    VT* un = Ub + (int64_t)(i + 1) * n;
    AT nacc = AT(0);
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        AT u = W[r];
#pragma unroll
        for (int q = 0; q < kMaxTrunc; ++q)
            if (q < nwin) u -= coef_sh[q] * ld_plain(Ub + (int64_t)(lo + q) * n + r);
        store_as(un + r, u);
        nacc += u * u;
    }
    nacc = block_sum(nacc, red);
    if (threadIdx.x == 0) normpart[b] = nacc;
}

// ---------------------------------------------------------------------------------------------------------------
// Sketched QR update of column i (one CTA).
__global__ void __launch_bounds__(512)
    k_inner_qr(int s, int m, int i, const double* __restrict__ C, double* __restrict__ Q, double* __restrict__ R,
               double* __restrict__ d, double* __restrict__ e, double* __restrict__ rho,
               CycleState* __restrict__ cyc) {
    extern __shared__ double qsm[];
    double* p = qsm;          // [s]
    double* a = qsm + s;      // [i] projection coefficients
    __shared__ double red[32];
    __shared__ int stop_sh;
    if (threadIdx.x == 0) stop_sh = cyc->stopped;
    __syncthreads();
    if (stop_sh) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = threadIdx.x; r < s; r += blockDim.x) p[r] = C[(int64_t)i * s + r];
    for (int l = threadIdx.x; l < i; l += blockDim.x) R[(int64_t)i * m + l] = 0.0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int l = warp; l < i; l += nw) {
            double acc = 0.0;
            const double* ql = Q + (int64_t)l * s;
            for (int r = lane; r < s; r += 32) acc += ql[r] * p[r];
            acc = warp_sum(acc);
            if (lane == 0) a[l] = acc;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < s; r += blockDim.x) {
            double v = p[r];
            for (int l = 0; l < i; ++l) v -= a[l] * Q[(int64_t)l * s + r];
            p[r] = v;
        }
        for (int l = threadIdx.x; l < i; l += blockDim.x) R[(int64_t)i * m + l] += a[l];
        __syncthreads();
    }
    double nrm2 = 0.0;
    for (int r = threadIdx.x; r < s; r += blockDim.x) nrm2 += p[r] * p[r];
    const double rii = sqrt(block_sum(nrm2, red));
    const double dmax = fmax(cyc->dmax, rii);
    const double dmin = (i == 0) ? rii : fmin(cyc->dmin, rii);
    const double kappa = (dmin > 0.0) ? dmax / dmin : INFINITY;
    if (!(kappa <= cyc->cond_thr)) {  // C2 (also catches rii == 0 and NaN): drop column i
        __syncthreads();
        if (threadIdx.x == 0) {
            cyc->stopped = 1;
            cyc->k = i;
            cyc->reason = (i == 0) ? 5 : 2;
        }
        return;
    }
    const double inv = 1.0 / rii;
    double dacc = 0.0;
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        const double q = p[r] * inv;
        p[r] = q;
        Q[(int64_t)i * s + r] = q;
        dacc += q * e[r];
    }
    const double di = block_sum(dacc, red);
    double eacc = 0.0;
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        const double ev = e[r] - di * p[r];
        e[r] = ev;
        eacc += ev * ev;
    }
    const double rh = sqrt(block_sum(eacc, red));
    if (threadIdx.x == 0) {
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

// z = sum_{l<k} coef_l u_l in FP64.
template <typename VT>
__global__ void __launch_bounds__(256) k_inner_gemv(int n, const VT* __restrict__ Ub, const double* __restrict__ coef,
                                                    const CycleState* __restrict__ cyc, double* __restrict__ z) {
    __shared__ double cf[kMaxM];
    const int k = cyc->k;
    for (int l = threadIdx.x; l < k; l += blockDim.x) cf[l] = coef[l];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < k; ++l) acc += cf[l] * (double)ld_plain(Ub + (int64_t)l * n + r);
        z[r] = acc;
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

template <typename MT, typename VT, typename AT>
static void inner_spmv_t(const Plan& p, int i, const MT* val) {
    const size_t sm = (size_t)p.Bn * sizeof(AT);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_inner_spmv<VV, UU, MT, VT, AT>, sm),
                              k_inner_spmv<VV, UU, MT, VT, AT><<<p.nblk, 512, sm, p.st>>>(
                                 p.n, p.Bn, p.nblk, p.s, p.t, i, p.rp, p.col, val, (const VT*)p.U, (AT*)p.W,
                                 p.sigma, (const AT*)p.normpart, (AT*)p.hpart, (AT*)p.cpart, p.seg, p.ent, p.cyc)));
}

void launch_inner_spmv(const Plan& p, int i) {
    if (p.prec == kFP64) inner_spmv_t<double, double, double>(p, i, p.val);
    else if (p.prec == kFP32) inner_spmv_t<float, float, float>(p, i, p.val32);
    else inner_spmv_t<float, __nv_bfloat16, float>(p, i, p.val32);
    ++g_launches;
}

template <typename VT, typename AT>
static void inner_axpy_t(const Plan& p, int i, bool last) {
    k_inner_axpy<VT, AT><<<p.nblk, 512, 0, p.st>>>(p.n, p.Bn, p.nblk, p.s, p.t, i, last ? 1 : 0, p.sk_scale,
                                                   (VT*)p.U, (const AT*)p.W, p.sigma, (AT*)p.normpart,
                                                   (const AT*)p.hpart, (const AT*)p.cpart, p.C, p.hco, p.cyc);
}

void launch_inner_axpy(const Plan& p, int i, bool last) {
    if (p.prec == kFP64) inner_axpy_t<double, double>(p, i, last);
    else if (p.prec == kFP32) inner_axpy_t<float, float>(p, i, last);
    else inner_axpy_t<__nv_bfloat16, float>(p, i, last);
    ++g_launches;
}

void launch_inner_qr(const Plan& p, int i) {
    const size_t sm = (size_t)(p.s + p.m) * sizeof(double);
    k_inner_qr<<<1, 512, sm, p.st>>>(p.s, p.m, i, p.C, p.Q, p.R, p.d, p.e, p.rho, p.cyc);
    ++g_launches;
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
