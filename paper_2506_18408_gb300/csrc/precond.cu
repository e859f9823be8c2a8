// Zero-fill incomplete LU (ILU(0)) right preconditioning in a multicolour order, on the device (the "-p" runs of
// Section 4: ILU(0) preconditioning; Table 1).
//
// The rows are ordered colour by colour (P: a greedy colouring of the pattern of A + A^T, computed once on the host
// when the handle's matrix is set up; no two coupled rows share a colour), and M = P^T L U P with L U the ILU(0)
// factorisation of the permuted matrix P A P^T.  Because rows of one colour are not coupled, the diagonal colour
// blocks of L are identities and those of U diagonal, so
//  * the factorisation is one pass per colour, every row of the colour independent (row r eliminates with the
//    finished rows k < r of earlier colours, in increasing k, dropping updates outside the pattern: the IKJ form), and
//  * M^{-1} u is one pass per colour forward (y_r = u_perm(r) - sum_{k<r} l_rk y_k) and one per colour backward
//    (z_r = (y_r - sum_{k>r} u_rk z_k) / u_rr, written back in the original order), one thread per row, coalesced
//    over the colour's consecutive rows, instead of a wavefront of ~3N dependent levels of the natural order.
// The permuted matrix is stored in CSR with sorted columns (permuted indices), its diagonal position per row, and
// the position of every entry in A's CSR, so new values of A refresh the factors without rebuilding the structure.
#include "kernels.h"

namespace sfg {

// lu[p] = val[src[p]]: the values of P A P^T in its own CSR order.
__global__ void k_ilu_gather(int64_t nnz, const int* __restrict__ src, const double* __restrict__ val,
                             double* __restrict__ lu) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) lu[p] = val[src[p]];
}

// ILU(0) of the rows [r0, r1) of one colour, one thread per row: for each entry (r, k) with k < r (earlier colours,
// already final), l_rk = a_rk / u_kk, then a_rj -= l_rk u_kj for the entries j > k that row r and row k both hold
// (a merge of the two sorted rows).  A zero pivot sets *bad.
__global__ void k_ilu0_colour(int r0, int r1, const int* __restrict__ rp, const int* __restrict__ col,
                              const int* __restrict__ diag, double* __restrict__ lu, int* __restrict__ bad) {
    const int r = r0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= r1) return;
    const int a = rp[r], e = rp[r + 1], dr = diag[r];
    for (int p = a; p < dr; ++p) {
        const int k = col[p];
        const double ukk = lu[diag[k]];
        if (ukk == 0.0) {
            atomicOr(bad, 1);
            return;
        }
        const double l = lu[p] / ukk;
        lu[p] = l;
        int q = p + 1;                             // row r's entries after column k
        int s = diag[k] + 1;                       // row k's entries after its diagonal
        const int se = rp[k + 1];
        while (q < e && s < se) {
            const int cq = col[q], cs = col[s];
            if (cq == cs) {
                lu[q] -= l * lu[s];
                ++q;
                ++s;
            } else if (cq < cs) {
                ++q;
            } else {
                ++s;
            }
        }
    }
    if (lu[dr] == 0.0) atomicOr(bad, 1);
}

// Whether the cycle of the plan's single problem has stopped before step i (nothing of step i is used then).
__device__ __forceinline__ bool ilu_idle(const Plan& P, int i) {
    if (i < 0) return false;
    const CycleState* c = P.cyc;
    return c->stopped || c->brk_step <= i || (P.pflag[0] & 1);
}

// Forward pass over the rows [r0, r1) of one colour: y_r = u[perm[r]] - sum_{k < r} l_rk y_k.
__global__ void k_ilu_fwd(const Plan P, int i, int r0, int r1, const double* __restrict__ u,
                          double* __restrict__ y) {
    if (ilu_idle(P, i)) return;
    const IluDev& I = P.ilu;
    const int r = r0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= r1) return;
    const int a = I.rp[r], dr = I.diag[r];
    double v = u[I.perm[r]];
    for (int p = a; p < dr; ++p) v -= I.lu[p] * y[I.col[p]];
    y[r] = v;
}

// Backward pass over the rows [r0, r1) of one colour: z_r = (y_r - sum_{k > r} u_rk z_k) / u_rr, and
// out[perm[r]] = z_r (the original order).
__global__ void k_ilu_bwd(const Plan P, int i, int r0, int r1, const double* __restrict__ y,
                          double* __restrict__ zp, double* __restrict__ out) {
    if (ilu_idle(P, i)) return;
    const IluDev& I = P.ilu;
    const int r = r0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= r1) return;
    const int dr = I.diag[r], e = I.rp[r + 1];
    double v = y[r];
    for (int p = dr + 1; p < e; ++p) v -= I.lu[p] * zp[I.col[p]];
    v /= I.lu[dr];
    zp[r] = v;
    out[I.perm[r]] = v;
}

cudaError_t launch_ilu_factor(const IluHost& H, const double* val, int* bad, cudaStream_t st) {
    const IluDev& I = H.dev;
    k_ilu_gather<<<(unsigned)((H.nnz + 255) / 256), 256, 0, st>>>(H.nnz, H.src, val, I.lu);
    for (int c = 0; c < H.ncol; ++c) {
        const int r0 = H.starts[c], r1 = H.starts[c + 1];
        if (r1 > r0) k_ilu0_colour<<<(unsigned)((r1 - r0 + 255) / 256), 256, 0, st>>>(r0, r1, I.rp, I.col, I.diag, I.lu, bad);
    }
    g_launches += 1 + H.ncol;
    return cudaGetLastError();
}

void launch_ilu_apply(const Plan& P, int i, const double* u, double* out) {
    const IluHost& H = *P.ilu_host;
    const IluDev& I = H.dev;
    for (int c = 0; c < H.ncol; ++c) {
        const int r0 = H.starts[c], r1 = H.starts[c + 1];
        if (r1 > r0) k_ilu_fwd<<<(unsigned)((r1 - r0 + 255) / 256), 256, 0, P.st>>>(P, i, r0, r1, u, I.y);
    }
    for (int c = H.ncol - 1; c >= 0; --c) {
        const int r0 = H.starts[c], r1 = H.starts[c + 1];
        if (r1 > r0) k_ilu_bwd<<<(unsigned)((r1 - r0 + 255) / 256), 256, 0, P.st>>>(P, i, r0, r1, I.y, I.zp, out);
    }
    g_launches += 2 * H.ncol;
}

}  // namespace sfg
