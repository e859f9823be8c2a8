// Host-side launchers of the sketched-FGMRES kernels, and the device-pointer plan they operate on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sfg {

enum Precision { kFP64 = 0, kFP32 = 1, kBF16 = 2 };

// Everything a kernel needs, as plain device pointers and sizes (owned by the solver handle).
struct Plan {
    // matrix (CSR, int32 indices)
    int n = 0;
    int64_t nnz = 0;
    const int* rp = nullptr;
    const int* col = nullptr;
    const double* val = nullptr;
    const float* val32 = nullptr;  // FP32 copy (inner FP32/BF16 modes)
    int vec = 8;                   // SpMV lanes per row (1 = one thread per row)

    // row blocks (shared by all fused kernels and by the sketch gather lists)
    int Bn = 0, nblk = 0;

    // sketch: per (row block b, sketch row r) the segment seg[b*s + r] .. seg[b*s + r + 1] of `ent`, each entry a
    // 15-bit row offset inside block b plus a sign bit (0x8000 = negative)
    int s = 0, zeta = 0, kind = 0;
    const int* seg = nullptr;
    const uint16_t* ent = nullptr;
    double sk_scale = 1.0;
    int sk_headroom = 0;  // extra right shift of the FP64 fixed-point sketch terms (long gather lists)

    // inner cycle
    int prec = kFP64, m = 0, t = 0;
    void* U = nullptr;         // basis storage, (m+1) columns of n (VT); column l = u_l, b_l = sigma[l] * u_l
    void* W = nullptr;         // w = A b_i (AT[n])
    double* sigma = nullptr;   // [m+1] 1/||u_l||
    void* normpart = nullptr;  // AT[2 * nblk], double-buffered by step parity
    void* hpart = nullptr;     // AT[nblk * kMaxTrunc]
    void* cpart = nullptr;     // AT[nblk * s]
    double* C = nullptr;       // [m * s]  S A b_i
    double* Q = nullptr;       // [m * s]
    double* R = nullptr;       // [m * m]  column-major, R[i*m + l] = R_{l,i}
    double* d = nullptr;       // [m]      q_l^T (running sketched residual)
    double* e = nullptr;       // [s]      running sketched residual S v - Q Q^T S v
    double* c0 = nullptr;      // [s]      S v
    double* rho = nullptr;     // [m]
    double* y = nullptr;       // [m]
    double* coef = nullptr;    // [m]      y_l * sigma_l
    double* hco = nullptr;     // [m * kMaxTrunc] truncated-Arnoldi coefficients
    CycleState* cyc = nullptr;

    // outer FGMRES
    int jmax = 0;
    double* Vb = nullptr;      // [(jmax+1) * n] unnormalised outer basis, v_l = nu[l] * Vb_l
    double* Z = nullptr;       // [jmax * n]
    double* nu = nullptr;      // [jmax+1]
    double* Wo = nullptr;      // [n] outer work vector
    double* opart = nullptr;   // [nblk * (jmax+1)]
    double* npart = nullptr;   // [nblk] (FP64 norm partials of outer / residual kernels)
    double* npart2 = nullptr;  // [nblk]
    double* h1 = nullptr;      // [jmax+1]
    double* h2 = nullptr;      // [jmax+1]
    double* H = nullptr;       // [(jmax+1) * jmax] column-major, H[j*(jmax+1) + l] = h_{l,j}
    double* cs = nullptr;      // [jmax]
    double* sn = nullptr;      // [jmax]
    double* g = nullptr;       // [jmax+1]
    double* yo = nullptr;      // [jmax]
    double* est_hist = nullptr;   // [jmax]
    double* ffom_hist = nullptr;  // [jmax]
    int* k_hist = nullptr;        // [jmax]
    int* reason_hist = nullptr;   // [jmax]
    OuterState* ost = nullptr;

    cudaStream_t st = nullptr;
};

// ---- sketch (sketch.cu) ----
void launch_sketch_pattern(const Plan& p, int n, int s, int zeta, int kind, uint64_t seed, int* rows, int8_t* neg,
                           cudaStream_t st);
// Gather lists in two steps: counts (int[nblk*s], zeroed by the caller) and seg (int[nblk*s + 1], list starts with
// lengths padded to multiples of 8); then, once the caller has read seg[nblk*s] = total and allocated
// ent (uint16[total + 8]), the fill (padding entries point at the zero slot Bn of each block).
void launch_sketch_count(int n, int s, int zeta, int Bn, int nblk, const int* rows, int* counts, int* seg,
                         cudaStream_t st);
void launch_sketch_fill(int n, int s, int zeta, int Bn, int nblk, const int* rows, const int8_t* neg,
                        const int* seg, uint16_t* ent, int64_t total, cudaStream_t st);
// part[nblk*s] = per-block sketch sums of (xscale * x), optionally storing (VT)(xscale*x) into dst
void launch_sketch_partials(const Plan& p, const double* x, const double* xscale_dev, void* dst, void* part);
// out[r] = sk_scale * sum_b part[b*s + r]; out2 (optional) gets the same values
void launch_sketch_reduce(const Plan& p, const void* part, double* out, double* out2);

// ---- inner cycle (inner.cu) ----
// resets the cycle state (j < 0: no outer solve, C3 off), u_0 = vscale * v, c0 = S u_0, e = c0
void launch_cycle_start(const Plan& p, int j, const double* v, const double* vscale_dev, int c3_on, double cond_thr);
void launch_inner_spmv(const Plan& p, int i);
void launch_inner_axpy(const Plan& p, int i, bool last);
cudaError_t launch_inner_qr(const Plan& p, int i, cudaStream_t st);  // cluster launch on stream st
void launch_inner_finish(const Plan& p, double* z);  // y = R^{-1} d, z = sum_l y_l b_l (FP64)
void launch_export_basis(const Plan& p, double* out, int count);  // out[:, l] = sigma_l * u_l (FP64)

// ---- outer FGMRES and helpers (outer.cu) ----
// rb = b - A x (x may be NULL = 0), npart/npart2 partials of ||rb||^2 and ||b||^2; rb may be NULL
void launch_residual(const Plan& p, const double* b, const double* x, double* rb);
void launch_init_state(const Plan& p, double tol, int jmax);  // beta, ||b||, nu_0 from npart/npart2
void launch_outer_step(const Plan& p, int j);                  // w = A z_j, CGS2 against v_0..v_j, Givens update
void launch_final_x(const Plan& p, int J, const double* x0, double* x);  // y = R^{-1} g, x = x0 + Z y
void launch_true_residual_reduce(const Plan& p);               // ost->true_res2 from npart
void launch_spmv_f64(const Plan& p, const double* x, double* y);

// Raise the dynamic shared-memory limit of kernel `func` to at least `bytes` (cached per kernel).
void set_smem(const void* func, size_t bytes);

// ---- transpose and pattern gradient (transpose.cu) ----
// counts: int[n] zeroed by the caller; rpT int[n+1]; colT, srcT int[nnz]; maxlen int (zeroed) gets the longest row
void launch_transpose(int n, int64_t nnz, const int* rp, const int* col, int* counts, int* rpT, int* colT,
                      int* srcT, int* maxlen, cudaStream_t st);
void launch_gather_vals(int64_t nnz, const int* src, const double* val, double* out, cudaStream_t st);
void launch_pattern_outer(int n, const int* rp, const int* col, const double* u, const double* v, double alpha,
                          double* out, cudaStream_t st);

// launch counter (incremented by every launcher)
extern thread_local int64_t g_launches;

}  // namespace sfg
