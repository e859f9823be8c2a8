// Outer FGMRES (Algorithm 1) on the device for every problem of a batch, FP64 throughout.
//
// Outer step j:  w = A z_j (fused with the first batch of dot products v_l^T w), two classical Gram-Schmidt passes
// against v_0..v_j (the reorthogonalised form of the orthogonalisation loop of Algorithm 1), h_{j+1,j} = ||w||,
// v_{j+1} = w / h_{j+1,j} (stored unnormalised with its scale nu), then one Givens rotation of the Hessenberg
// column, which gives the FGMRES residual estimate |g_{j+1}| and the FFOM residual |g_{j+1}| / |c_j| (Eq. 4: the
// FFOM residual is h_{j+1,j} |gamma_j|; in rotated form this is the FGMRES residual divided by the cosine of the
// last rotation).  The FFOM residual feeds rule C3 of the next inner cycle through the bound of Eq. 5.
// Row-block kernels skip the blocks of problems that are done; per-problem kernels reduce their problem's block
// partials in block order, so every sum has a fixed order.
#include "kernels.h"
#include "spmv.cuh"

#include <algorithm>

namespace sfg {

__device__ __forceinline__ bool outer_idle(const Plan& P, int p) { return (P.pflag[p] & 1) != 0; }

// rb = b - A x (x may be null: rb = b); npart[b] = ||rb||^2 over the block, npart2[b] = ||b||^2 over the block.
template <int V, int U>
__global__ void __launch_bounds__(512, 2)
    k_residual(const Plan P, const double* __restrict__ bv, const double* __restrict__ x, double* __restrict__ rb,
               int only_final) {
    extern __shared__ double axb[];
    __shared__ double red[32];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    const int fl = P.pflag[bi.prob];
    if (only_final ? !(fl & 2) : (fl & 1)) return;
    if (x) {
        const int m0 = bi.v0 - bi.cs;
        int n0, n01;
        block_bins(P, bi, n0, n01);
        spmv_rows_to_smem<V, U, double, double, double>(P.rp, (V == 0 && P.brp) ? P.bcol : P.col, (V == 0 && P.brp) ? P.bval : P.val, x + bi.cs, m0, m0 + bi.len, axb, P.perm,
                                                        n0, n01, V == 0 ? P.brp : nullptr);
        __syncthreads();
    }
    double a1 = 0.0, a2 = 0.0;
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) {
        const int r = bi.v0 + k;
        const double bb = bv[r];
        const double rr = x ? bb - axb[k] : bb;
        if (rb) rb[r] = rr;
        a1 += rr * rr;
        a2 += bb * bb;
    }
    a1 = block_sum(a1, red);
    a2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        P.npart[b] = a1;
        P.npart2[b] = a2;
    }
}

void launch_residual(const Plan& p, const double* b, const double* x, double* rb, bool only_final) {
    const size_t sm = x ? (size_t)p.Bn * sizeof(double) : 0;
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_residual<VV, UU>, sm),
                              k_residual<VV, UU><<<p.nblk, 512, sm, p.st>>>(p, b, x, rb, only_final ? 1 : 0)));
    ++g_launches;
}

// Per problem (one warp each): beta = ||r0||, ||b||, tol * ||b||, nu_0 = 1/beta, g_0 = beta.
__global__ void k_init_state(const Plan P, double tol) {
    const int p = blockIdx.x, lane = threadIdx.x;
    double a1 = 0.0, a2 = 0.0;
    for (int q = P.prob_b0[p] + lane; q < P.prob_b0[p + 1]; q += 32) {
        a1 += P.npart[q];
        a2 += P.npart2[q];
    }
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
        OuterState* ost = P.ost + p;
        const double beta = sqrt(a1), bn = sqrt(a2);
        ost->j = 0;
        ost->conv_est = 0;
        ost->breakdown = 0;
        ost->nan = (!isfinite(a1) || !isfinite(a2)) ? 1 : 0;
        ost->sync_fail = 0;
        ost->beta = beta;
        ost->bnorm = bn;
        ost->est = beta;
        ost->ffom = beta;
        ost->true_res2 = a1;
        ost->tol_abs = tol * bn;
        const int64_t o = (int64_t)p * (P.jmax + 1);
        P.nu[o] = (beta > 0.0) ? 1.0 / beta : 0.0;
        P.g[o] = beta;
    }
}

void launch_init_state(const Plan& p, double tol) {
    k_init_state<<<p.P, 32, 0, p.st>>>(p, tol);
    ++g_launches;
}

// Per problem flagged "finalise now": ost[p].true_res2 = sum of its blocks' npart.
__global__ void k_true_res(const Plan P) {
    const int p = blockIdx.x;
    if (!(P.pflag[p] & 2)) return;
    double a = 0.0;
    for (int q = P.prob_b0[p] + threadIdx.x; q < P.prob_b0[p + 1]; q += 32) a += P.npart[q];
    a = warp_sum(a);
    if (threadIdx.x == 0) P.ost[p].true_res2 = a;
}

void launch_true_residual_reduce(const Plan& p) {
    k_true_res<<<p.P, 32, 0, p.st>>>(p);
    ++g_launches;
}

// Dots of the block's part of v_0..v_j with the block vector wb (smem): opart[b*ldo + l], one warp per column.
__device__ __forceinline__ void block_dots(const Plan& P, const BlockInfo& bi, int b, int j,
                                           const double* __restrict__ wb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ldo = P.jmax + 1;
    for (int l = warp; l <= j; l += nw) {
        const double* vl = P.Vb + (int64_t)l * P.N + bi.v0;
        double acc = 0.0;
        for (int k = lane; k < bi.len; k += 32) acc += vl[k] * wb[k];
        acc = warp_sum(acc);
        if (lane == 0) P.opart[(int64_t)b * ldo + l] = acc;
    }
}

// w = A z_j into smem and Wo; opart[b*ldo + l] = Vb_l(block) . w(block) for l <= j.
template <int V, int U>
__global__ void __launch_bounds__(512, 2) k_outer_spmv(const Plan P, int j) {
    extern __shared__ double wb[];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    if (outer_idle(P, bi.prob)) return;
    const double* z = P.Z + (int64_t)j * P.N;
    const int m0 = bi.v0 - bi.cs;
    int n0, n01;
    block_bins(P, bi, n0, n01);
    spmv_rows_to_smem<V, U, double, double, double>(P.rp, (V == 0 && P.brp) ? P.bcol : P.col, (V == 0 && P.brp) ? P.bval : P.val, z + bi.cs, m0, m0 + bi.len, wb, P.perm, n0,
                                                    n01, V == 0 ? P.brp : nullptr);
    __syncthreads();
    // the true residual of inner cycle j, r_hat_j = v_j - A z_j (v_j = nu_j Vb_j), for the bound of Eq. 5: its
    // block partial of ||r_hat_j||^2 goes to npart2 (free during outer steps)
    const double nuj = P.nu[(int64_t)bi.prob * (P.jmax + 1) + j];
    const double* vj = P.Vb + (int64_t)j * P.N;
    double r2 = 0.0;
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) {
        const double w = wb[k];
        P.Wo[bi.v0 + k] = w;
        const double rr = nuj * vj[bi.v0 + k] - w;
        r2 += rr * rr;
    }
    block_dots(P, bi, b, j, wb);
    __shared__ double red[32];
    r2 = block_sum(r2, red);
    if (threadIdx.x == 0) P.npart2[b] = r2;
}

// out[p*ldo + l] = nu[p][l] * sum over the blocks of problem p of opart[b*ldo + l]  (one warp per (p, l)).
__global__ void k_reduce_cols(const Plan P, int ncols, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= (int64_t)P.P * ncols) return;
    const int p = (int)(w / ncols), l = (int)(w % ncols);
    if (outer_idle(P, p)) return;
    const int ldo = P.jmax + 1;
    double acc = 0.0;
    for (int q = P.prob_b0[p] + lane; q < P.prob_b0[p + 1]; q += 32) acc += P.opart[(int64_t)q * ldo + l];
    acc = warp_sum(acc);
    if (lane == 0) out[(int64_t)p * ldo + l] = P.nu[(int64_t)p * ldo + l] * acc;
}

// One classical Gram-Schmidt subtraction w <- w - sum_{l<=j} h_l v_l with v_l = nu_l Vb_l.
//  final == 0: result back into Wo and the next pass's dots into opart
//  final == 1: result into Vb_{j+1} (unnormalised) and ||w||^2 partials into npart
__global__ void __launch_bounds__(512, 2)
    k_outer_cgs(const Plan P, int j, int final_pass, const double* __restrict__ h) {
    extern __shared__ double sm[];
    double* cf = sm;            // [j+1]
    double* wb = sm + (j + 1);  // [Bn]
    __shared__ double red[32];
    const int b = blockIdx.x;
    const BlockInfo bi = block_info(P, b);
    const int p = bi.prob;
    if (outer_idle(P, p)) return;
    const int N = P.N;
    const int64_t o = (int64_t)p * (P.jmax + 1);
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cf[l] = h[o + l] * P.nu[o + l];
    __syncthreads();
    double* dst = P.Vb + (int64_t)(j + 1) * N;
    double nacc = 0.0;
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) {
        const int r = bi.v0 + k;
        double w = P.Wo[r];
        for (int l = 0; l <= j; ++l) w -= cf[l] * P.Vb[(int64_t)l * N + r];
        if (final_pass) {
            dst[r] = w;
            nacc += w * w;
        } else {
            P.Wo[r] = w;
            wb[k] = w;
        }
    }
    if (final_pass) {
        nacc = block_sum(nacc, red);
        if (threadIdx.x == 0) P.npart[b] = nacc;
        return;
    }
    __syncthreads();
    block_dots(P, bi, b, j, wb);
}

// Per problem (one warp): Hessenberg column j = h1 + h2 (and h_{j+1,j} = ||w||), Givens update, residual
// estimates, histories.
__global__ void k_outer_givens(const Plan P, int j) {
    const int p = blockIdx.x, lane = threadIdx.x;
    if (outer_idle(P, p)) return;
    const int ldo = P.jmax + 1, J = P.jmax;
    double a = 0.0, ar = 0.0;
    for (int q = P.prob_b0[p] + lane; q < P.prob_b0[p + 1]; q += 32) {
        a += P.npart[q];
        ar += P.npart2[q];
    }
    a = warp_sum(a);
    ar = warp_sum(ar);
    if (lane != 0) return;
    OuterState* ost = P.ost + p;
    const CycleState* cyc = P.cyc + p;
    const int64_t oh = (int64_t)p * J, og = (int64_t)p * ldo;
    P.ires_hist[oh + j] = sqrt(ar);  // ||v_j - A z_j||: the factor ||r_hat_j|| of the bound of Eq. 5
    P.rho_hist[oh + j] = cyc->rho;   // the cycle's sketched estimate of it (rule C3)
    if (P.gsync && P.gsync[1]) {  // the inner cycle's grid-wide wait gave up: its results are not valid
        ost->sync_fail = 1;
        ost->nan = 1;
    }
    P.k_hist[oh + j] = cyc->k;
    P.reason_hist[oh + j] = cyc->reason;
    if (cyc->k == 0) {  // inner cycle produced no correction
        ost->breakdown = 2;
        return;
    }
    if (cyc->reason == 6) ost->nan = 1;
    const double* h1 = P.h1 + og;
    const double* h2 = P.h2 + og;
    double* cs = P.cs + oh;
    double* sn = P.sn + oh;
    double* g = P.g + og;
    const double hn = sqrt(a);
    double* colj = P.H + og * J + (int64_t)j * ldo;
    for (int l = 0; l <= j; ++l) colj[l] = h1[l] + h2[l];
    colj[j + 1] = hn;
    for (int l = 0; l < j; ++l) {
        const double x0 = colj[l], x1 = colj[l + 1];
        colj[l] = cs[l] * x0 + sn[l] * x1;
        colj[l + 1] = -sn[l] * x0 + cs[l] * x1;
    }
    const double aa = colj[j], bb = colj[j + 1];
    const double r = hypot(aa, bb);
    double c = 1.0, s = 0.0;
    if (r > 0.0) {
        c = aa / r;
        s = bb / r;
    }
    cs[j] = c;
    sn[j] = s;
    colj[j] = r;
    colj[j + 1] = 0.0;
    const double gj = g[j];
    g[j] = c * gj;
    g[j + 1] = -s * gj;
    const double est = fabs(g[j + 1]);
    const double ffom = (c != 0.0) ? est / fabs(c) : INFINITY;
    P.nu[og + j + 1] = (hn > 0.0) ? 1.0 / hn : 0.0;
    if (P.outer_variant == 1 && c == 0.0) {  // FFOM: the square system of this step is singular; keep step j's x
        ost->breakdown = 2;
        return;
    }
    const double e = (P.outer_variant == 1) ? ffom : est;  // the variant's residual estimate
    ost->j = j + 1;
    ost->est = e;
    ost->ffom = ffom;
    ost->breakdown = (hn == 0.0) ? 1 : 0;
    ost->conv_est = (e <= ost->tol_abs) ? 1 : 0;
    if (!isfinite(est) || !isfinite(hn) || !isfinite(r)) ost->nan = 1;
    P.est_hist[oh + j] = e / ost->bnorm;
    P.ffom_hist[oh + j] = ffom / ost->bnorm;
}

void launch_outer_step(const Plan& p, int j) {
    const size_t sm = (size_t)p.Bn * sizeof(double);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_outer_spmv<VV, UU>, sm),
                              k_outer_spmv<VV, UU><<<p.nblk, 512, sm, p.st>>>(p, j)));
    const int ncols = j + 1, wpb = 8;
    const int rgrid = (int)(((int64_t)p.P * ncols + wpb - 1) / wpb);
    k_reduce_cols<<<rgrid, 32 * wpb, 0, p.st>>>(p, ncols, p.h1);
    const size_t sm2 = (size_t)(p.Bn + j + 1) * sizeof(double);
    set_smem((const void*)k_outer_cgs, sm2);
    k_outer_cgs<<<p.nblk, 512, sm2, p.st>>>(p, j, 0, p.h1);
    k_reduce_cols<<<rgrid, 32 * wpb, 0, p.st>>>(p, ncols, p.h2);
    k_outer_cgs<<<p.nblk, 512, (size_t)(j + 1) * sizeof(double), p.st>>>(p, j, 1, p.h2);
    k_outer_givens<<<p.P, 32, 0, p.st>>>(p, j);
    g_launches += 6;
}

// Per problem flagged "finalise now" (one warp): y = R^{-1} g over the rotated J x J triangle, J = the problem's
// outer iteration count.
__global__ void k_final_y(const Plan P) {
    extern __shared__ double rhs[];
    const int p = blockIdx.x;
    if (!(P.pflag[p] & 2)) return;
    const int ldo = P.jmax + 1, J = P.ost[p].j;
    const double* H = P.H + (int64_t)p * ldo * P.jmax;
    const double* g = P.g + (int64_t)p * ldo;
    double* y = P.yo + (int64_t)p * P.jmax;
    const int lane = threadIdx.x;
    // FFOM: the square system before the last rotation (c, s) has last diagonal c r_JJ and last right-hand side
    // g_J / c; the rows above are those of R
    const double cl = (P.outer_variant == 1 && J > 0) ? P.cs[(int64_t)p * P.jmax + J - 1] : 1.0;
    for (int l = lane; l < J; l += 32) rhs[l] = (l == J - 1) ? g[l] / cl : g[l];
    __syncwarp();
    for (int l = J - 1; l >= 0; --l) {
        const double yl = rhs[l] / (H[(int64_t)l * ldo + l] * ((l == J - 1) ? cl : 1.0));
        for (int q = lane; q < l; q += 32) rhs[q] -= H[(int64_t)l * ldo + q] * yl;
        if (lane == 0) y[l] = yl;
        __syncwarp();
    }
}

// x = x0 + Z y over the blocks of flagged problems.
__global__ void __launch_bounds__(256) k_final_x(const Plan P, const double* __restrict__ x0,
                                                 double* __restrict__ x) {
    __shared__ double yy[kMaxM];
    const BlockInfo bi = block_info(P, blockIdx.x);
    const int p = bi.prob;
    if (!(P.pflag[p] & 2)) return;
    const int J = P.ost[p].j, N = P.N;
    for (int l = threadIdx.x; l < J; l += blockDim.x) yy[l] = P.yo[(int64_t)p * P.jmax + l];
    __syncthreads();
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) {
        const int64_t r = bi.v0 + k;
        double acc = x0 ? x0[r] : 0.0;
        for (int l = 0; l < J; ++l) acc += yy[l] * P.Z[(int64_t)l * N + r];
        x[r] = acc;
    }
}

void launch_final_x(const Plan& p, int J, const double* x0, double* x) {
    k_final_y<<<p.P, 32, (size_t)std::max(J, 1) * sizeof(double), p.st>>>(p);
    k_final_x<<<p.nblk, 256, 0, p.st>>>(p, x0, x);
    g_launches += 2;
}

template <int V, int U>
__global__ void __launch_bounds__(512, 2)
    k_spmv_plain(const Plan P, const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ double yb[];
    const BlockInfo bi = block_info(P, blockIdx.x);
    const int m0 = bi.v0 - bi.cs;
    int n0, n01;
    block_bins(P, bi, n0, n01);
    spmv_rows_to_smem<V, U, double, double, double>(P.rp, (V == 0 && P.brp) ? P.bcol : P.col, (V == 0 && P.brp) ? P.bval : P.val, x + bi.cs, m0, m0 + bi.len, yb, P.perm, n0,
                                                    n01, V == 0 ? P.brp : nullptr);
    __syncthreads();
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) y[bi.v0 + k] = yb[k];
}

void launch_spmv_f64(const Plan& p, const double* x, double* y) {
    const size_t sm = (size_t)p.Bn * sizeof(double);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_spmv_plain<VV, UU>, sm),
                              k_spmv_plain<VV, UU><<<p.nblk, 512, sm, p.st>>>(p, x, y)));
    ++g_launches;
}

}  // namespace sfg
