// Outer FGMRES (Algorithm 1) on the device, FP64 throughout.
//
// Outer step j:  w = A z_j (fused with the first batch of dot products v_l^T w), two classical Gram-Schmidt passes
// against v_0..v_j (the reorthogonalised form of the orthogonalisation loop of Algorithm 1), h_{j+1,j} = ||w||,
// v_{j+1} = w / h_{j+1,j} (stored unnormalised with its scale nu), then one Givens rotation of the Hessenberg
// column, which gives the FGMRES residual estimate |g_{j+1}| and the FFOM residual |g_{j+1}| / |c_j| (Eq. 4: the
// FFOM residual is h_{j+1,j} |gamma_j|; in rotated form this is the FGMRES residual divided by the cosine of the
// last rotation).  The FFOM residual feeds rule C3 of the next inner cycle through the bound of Eq. 5.
#include "kernels.h"
#include "spmv.cuh"

#include <algorithm>

namespace sfg {

// rb = b - A x (x may be null: rb = b); npart[b] = ||rb||^2 over the block, npart2[b] = ||b||^2 over the block.
template <int V, int U>
__global__ void __launch_bounds__(512, 2)
    k_residual(int n, int Bn, const int* __restrict__ rp, const int* __restrict__ col,
               const double* __restrict__ val, const double* __restrict__ bv, const double* __restrict__ x,
               double* __restrict__ rb, double* __restrict__ npart, double* __restrict__ npart2) {
    extern __shared__ double axb[];
    __shared__ double red[32];
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    if (x) {
        spmv_rows_to_smem<V, U, double, double, double>(rp, col, val, x, r0, r1, axb);
        __syncthreads();
    }
    double a1 = 0.0, a2 = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const double bb = bv[r];
        const double rr = x ? bb - axb[r - r0] : bb;
        if (rb) rb[r] = rr;
        a1 += rr * rr;
        a2 += bb * bb;
    }
    a1 = block_sum(a1, red);
    a2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        npart[b] = a1;
        npart2[b] = a2;
    }
}

void launch_residual(const Plan& p, const double* b, const double* x, double* rb) {
    const size_t sm = (size_t)p.Bn * sizeof(double);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_residual<VV, UU>, sm), k_residual<VV, UU><<<p.nblk, 512, sm, p.st>>>(p.n, p.Bn, p.rp, p.col, p.val, b, x,
                                                                          rb, p.npart, p.npart2)));
    ++g_launches;
}

__global__ void k_init_state(int nblk, const double* __restrict__ npart, const double* __restrict__ npart2,
                             double tol, OuterState* ost, double* nu) {
    const int lane = threadIdx.x;
    double a1 = 0.0, a2 = 0.0;
    for (int q = lane; q < nblk; q += 32) {
        a1 += npart[q];
        a2 += npart2[q];
    }
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
        const double beta = sqrt(a1), bn = sqrt(a2);
        ost->j = 0;
        ost->conv_est = 0;
        ost->breakdown = 0;
        ost->nan = (!isfinite(a1) || !isfinite(a2)) ? 1 : 0;
        ost->beta = beta;
        ost->bnorm = bn;
        ost->est = beta;
        ost->ffom = beta;
        ost->true_res2 = a1;
        ost->tol_abs = tol * bn;
        nu[0] = (beta > 0.0) ? 1.0 / beta : 0.0;
    }
}

void launch_init_state(const Plan& p, double tol, int) {
    k_init_state<<<1, 32, 0, p.st>>>(p.nblk, p.npart, p.npart2, tol, p.ost, p.nu);
    ++g_launches;
}

__global__ void k_true_res(int nblk, const double* __restrict__ npart, OuterState* ost) {
    double a = 0.0;
    for (int q = threadIdx.x; q < nblk; q += 32) a += npart[q];
    a = warp_sum(a);
    if (threadIdx.x == 0) ost->true_res2 = a;
}

void launch_true_residual_reduce(const Plan& p) {
    k_true_res<<<1, 32, 0, p.st>>>(p.nblk, p.npart, p.ost);
    ++g_launches;
}

// w = A z into smem and Wo; opart[b*ldo + l] = Vb_l(block) . w(block) for l <= j.
template <int V, int U>
__global__ void __launch_bounds__(512, 2)
    k_outer_spmv(int n, int Bn, int j, int ldo, const int* __restrict__ rp, const int* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ z, const double* __restrict__ Vb,
                 double* __restrict__ Wo, double* __restrict__ opart) {
    extern __shared__ double wb[];
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    spmv_rows_to_smem<V, U, double, double, double>(rp, col, val, z, r0, r1, wb);
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) Wo[r] = wb[r - r0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l <= j; l += nw) {
        const double* vl = Vb + (int64_t)l * n;
        double acc = 0.0;
        for (int r = r0 + lane; r < r1; r += 32) acc += vl[r] * wb[r - r0];
        acc = warp_sum(acc);
        if (lane == 0) opart[(int64_t)b * ldo + l] = acc;
    }
}

// out[l] = nu[l] * sum_b opart[b*ldo + l] for l < ncols (one warp per column, fixed order)
__global__ void k_reduce_cols(int nblk, int ncols, int ldo, const double* __restrict__ opart,
                              const double* __restrict__ nu, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= ncols) return;
    double acc = 0.0;
    for (int q = lane; q < nblk; q += 32) acc += opart[(int64_t)q * ldo + l];
    acc = warp_sum(acc);
    if (lane == 0) out[l] = nu[l] * acc;
}

// One classical Gram-Schmidt subtraction w <- w - sum_{l<=j} h_l v_l with v_l = nu_l Vb_l.
//  final == 0: result back into Wo and the next pass's dots into opart
//  final == 1: result into dst (= Vb_{j+1}, unnormalised) and ||w||^2 partials into npart
__global__ void __launch_bounds__(512, 2)
    k_outer_cgs(int n, int Bn, int j, int ldo, int final_pass, const double* __restrict__ Vb,
                const double* __restrict__ nu, const double* __restrict__ h, double* __restrict__ Wo,
                double* __restrict__ opart, double* __restrict__ dst, double* __restrict__ npart) {
    extern __shared__ double sm[];
    double* cf = sm;              // [j+1]
    double* wb = sm + (j + 1);    // [Bn]
    __shared__ double red[32];
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cf[l] = h[l] * nu[l];
    __syncthreads();
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    double nacc = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double w = Wo[r];
        for (int l = 0; l <= j; ++l) w -= cf[l] * Vb[(int64_t)l * n + r];
        if (final_pass) {
            dst[r] = w;
            nacc += w * w;
        } else {
            Wo[r] = w;
            wb[r - r0] = w;
        }
    }
    if (final_pass) {
        nacc = block_sum(nacc, red);
        if (threadIdx.x == 0) npart[b] = nacc;
        return;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l <= j; l += nw) {
        const double* vl = Vb + (int64_t)l * n;
        double acc = 0.0;
        for (int r = r0 + lane; r < r1; r += 32) acc += vl[r] * wb[r - r0];
        acc = warp_sum(acc);
        if (lane == 0) opart[(int64_t)b * ldo + l] = acc;
    }
}

// Hessenberg column j = h1 + h2 (and h_{j+1,j} = ||w||), Givens update, residual estimates, histories.
__global__ void k_outer_givens(int j, int nblk, int ldH, const double* __restrict__ npart,
                               const double* __restrict__ h1, const double* __restrict__ h2, double* __restrict__ H,
                               double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                               double* __restrict__ nu, OuterState* ost, const CycleState* cyc,
                               double* __restrict__ est_hist, double* __restrict__ ffom_hist,
                               int* __restrict__ k_hist, int* __restrict__ reason_hist) {
    const int lane = threadIdx.x;
    double a = 0.0;
    for (int q = lane; q < nblk; q += 32) a += npart[q];
    a = warp_sum(a);
    if (lane != 0) return;
    k_hist[j] = cyc->k;
    reason_hist[j] = cyc->reason;
    if (cyc->k == 0) {  // inner cycle produced no correction
        ost->breakdown = 2;
        return;
    }
    if (cyc->reason == 6) ost->nan = 1;
    const double hn = sqrt(a);
    double* colj = H + (int64_t)j * ldH;
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
    nu[j + 1] = (hn > 0.0) ? 1.0 / hn : 0.0;
    ost->j = j + 1;
    ost->est = est;
    ost->ffom = ffom;
    ost->breakdown = (hn == 0.0) ? 1 : 0;
    ost->conv_est = (est <= ost->tol_abs) ? 1 : 0;
    if (!isfinite(est) || !isfinite(hn) || !isfinite(r)) ost->nan = 1;
    est_hist[j] = est / ost->bnorm;
    ffom_hist[j] = ffom / ost->bnorm;
}

__global__ void k_givens_init(double* g, const OuterState* ost) {
    if (threadIdx.x == 0) g[0] = ost->beta;
}

void launch_outer_step(const Plan& p, int j) {
    const int ldo = p.jmax + 1;
    const double* z = p.Z + (int64_t)j * p.n;
    if (j == 0) {
        k_givens_init<<<1, 32, 0, p.st>>>(p.g, p.ost);
        ++g_launches;
    }
    const size_t sm = (size_t)p.Bn * sizeof(double);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_outer_spmv<VV, UU>, sm), k_outer_spmv<VV, UU><<<p.nblk, 512, sm, p.st>>>(p.n, p.Bn, j, ldo, p.rp, p.col,
                                                                             p.val, z, p.Vb, p.Wo, p.opart)));
    const int ncols = j + 1, wpb = 8;
    const int rgrid = (ncols + wpb - 1) / wpb;
    k_reduce_cols<<<rgrid, 32 * wpb, 0, p.st>>>(p.nblk, ncols, ldo, p.opart, p.nu, p.h1);
    const size_t sm2 = (size_t)(p.Bn + j + 1) * sizeof(double);
    set_smem((const void*)k_outer_cgs, sm2);
    k_outer_cgs<<<p.nblk, 512, sm2, p.st>>>(p.n, p.Bn, j, ldo, 0, p.Vb, p.nu, p.h1, p.Wo, p.opart, nullptr,
                                             nullptr);
    k_reduce_cols<<<rgrid, 32 * wpb, 0, p.st>>>(p.nblk, ncols, ldo, p.opart, p.nu, p.h2);
    k_outer_cgs<<<p.nblk, 512, (size_t)(j + 1) * sizeof(double), p.st>>>(
        p.n, p.Bn, j, ldo, 1, p.Vb, p.nu, p.h2, p.Wo, nullptr, p.Vb + (int64_t)(j + 1) * p.n, p.npart);
    k_outer_givens<<<1, 32, 0, p.st>>>(j, p.nblk, ldo, p.npart, p.h1, p.h2, p.H, p.cs, p.sn, p.g, p.nu, p.ost,
                                       p.cyc, p.est_hist, p.ffom_hist, p.k_hist, p.reason_hist);
    g_launches += 6;
}

// y = R^{-1} g over the rotated J x J triangle (one warp).
__global__ void k_final_y(int J, int ldH, const double* __restrict__ H, const double* __restrict__ g,
                          double* __restrict__ y) {
    extern __shared__ double rhs[];
    const int lane = threadIdx.x;
    for (int l = lane; l < J; l += 32) rhs[l] = g[l];
    __syncwarp();
    for (int l = J - 1; l >= 0; --l) {
        const double yl = rhs[l] / H[(int64_t)l * ldH + l];
        for (int q = lane; q < l; q += 32) rhs[q] -= H[(int64_t)l * ldH + q] * yl;
        if (lane == 0) y[l] = yl;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_final_x(int n, int J, const double* __restrict__ Z,
                                                 const double* __restrict__ y, const double* __restrict__ x0,
                                                 double* __restrict__ x) {
    __shared__ double yy[1024];
    for (int l = threadIdx.x; l < J; l += blockDim.x) yy[l] = y[l];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = x0 ? x0[r] : 0.0;
        for (int l = 0; l < J; ++l) acc += yy[l] * Z[(int64_t)l * n + r];
        x[r] = acc;
    }
}

void launch_final_x(const Plan& p, int J, const double* x0, double* x) {
    k_final_y<<<1, 32, (size_t)std::max(J, 1) * sizeof(double), p.st>>>(J, p.jmax + 1, p.H, p.g, p.yo);
    const int th = 256;
    const int gr = (int)std::min<int64_t>(((int64_t)p.n + th - 1) / th, 152 * 8);
    k_final_x<<<gr, th, 0, p.st>>>(p.n, J, p.Z, p.yo, x0, x);
    g_launches += 2;
}

template <int V, int U>
__global__ void __launch_bounds__(512, 2)
    k_spmv_plain(int n, int Bn, const int* __restrict__ rp, const int* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ double yb[];
    const int b = blockIdx.x;
    const int r0 = b * Bn, r1 = min(n, r0 + Bn);
    spmv_rows_to_smem<V, U, double, double, double>(rp, col, val, x, r0, r1, yb);
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) y[r] = yb[r - r0];
}

void launch_spmv_f64(const Plan& p, const double* x, double* y) {
    const size_t sm = (size_t)p.Bn * sizeof(double);
    SFG_SPMV_DISPATCH(p.vec, (set_smem((const void*)k_spmv_plain<VV, UU>, sm), k_spmv_plain<VV, UU><<<p.nblk, 512, sm, p.st>>>(p.n, p.Bn, p.rp, p.col, p.val, x, y)));
    ++g_launches;
}

}  // namespace sfg
