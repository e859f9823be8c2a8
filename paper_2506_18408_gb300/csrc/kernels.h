// Host-side launchers of the sketched-FGMRES kernels, and the device-pointer plan they operate on.
//
// Every solve is a batch of independent *problems*: problem p is right-hand side r of system q (one system and one
// right-hand side for sfgmres_solve).  Each problem has its own inner cycle, outer FGMRES, stop rules and sketch
// vectors; all problems advance in lockstep (step i of cycle j) and a problem that has stopped is skipped.
// Vectors are concatenations over problems (problem p occupies rows prob_v0[p] .. prob_v0[p+1]); the systems' CSR
// matrices are concatenated block-diagonally (system q occupies matrix rows and columns moff_q .. moff_q + n_q).
// The rows of every problem are cut into row blocks of at most Bn rows that never straddle problems; block b is
// rows blk_v0[b] .. blk_v0[b] + blk_len[b] of the vectors, which are matrix rows of its system shifted by blk_cs[b]
// (vector index = matrix index + blk_cs[b]), so the right-hand sides of one system share one matrix and one set of
// sketch gather lists (list block blk_list[b]).  Kernels receive the Plan by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace sfg {

enum Precision { kFP64 = 0, kFP32 = 1, kBF16 = 2 };

// ILU(0) right preconditioner in a multicolour order (precond.cu): the permuted matrix P A P^T in CSR with sorted
// columns, its factors and work vectors (device pointers; a value member of the plan, so kernels read it directly).
struct IluDev {
    const int* rp = nullptr;    // [n+1]
    const int* col = nullptr;   // [nnz] columns (permuted indices), sorted within each row
    const int* diag = nullptr;  // [n] position of the diagonal entry in its row
    const int* perm = nullptr;  // [n] original index of permuted row r
    double* lu = nullptr;       // [nnz] L strictly below the diagonal (unit diagonal implied), U from the diagonal on
    double* y = nullptr;        // [n] forward-pass vector (permuted order)
    double* zp = nullptr;       // [n] backward-pass vector (permuted order)
};
// Host side of the preconditioner: the colour ranges the launchers loop over.
struct IluHost {
    int n = 0, ncol = 0;
    int64_t nnz = 0;
    std::vector<int> starts;   // [ncol + 1] first permuted row of each colour
    const int* src = nullptr;  // device [nnz]: position in A's CSR of every entry of P A P^T
    IluDev dev;
};

// Everything a kernel needs, as plain device pointers and sizes (owned by the solver handle).
struct Plan {
    // matrix (concatenated CSR, int32 indices, global column indices)
    int64_t nnz = 0;
    const int* rp = nullptr;
    const int* col = nullptr;
    const double* val = nullptr;
    const float* val32 = nullptr;  // FP32 copy (inner FP32/BF16 modes)
    int vec = 8;                   // SpMV lanes per row (1 = one thread per row, 0 = length-binned)
    // SELL-32 copy for the one-thread-per-row FP64 inner SpMV (vec == 1, FP64 inner cycles): slice widths as prefix
    // sums in units of 32 entries, per-lane row lengths, columns and values in slice order, and the first slice of
    // every list block
    const int* sl_off = nullptr;
    const uint8_t* sl_len = nullptr;
    const int* sl_col = nullptr;
    const double* sl_val = nullptr;
    const int* sl_base = nullptr;
    const uint16_t* perm = nullptr;  // length-binned SpMV: per matrix row block, its rows in length order
    // the length-binned SpMV's FP64 copy of A with each block's rows stored in that order (null: read the CSR
    // arrays through perm): row i of block L's order at brp[m0 + i] .. brp[m0 + i + 1] of bcol/bval
    const int* brp = nullptr;
    const int* bcol = nullptr;
    const double* bval = nullptr;
    const int* cls = nullptr;        // [2 * list blocks]: rows with <= 16 entries, rows with <= 64 entries

    // problems and row blocks
    int N = 0;                     // total vector length (sum over problems)
    int P = 0;                     // problems
    int nblk = 0;                  // row blocks over all problems
    int Bn = 0;                    // largest block
    const int* blk_v0 = nullptr;   // [nblk] first vector row
    const int* blk_len = nullptr;  // [nblk] rows
    const int* blk_cs = nullptr;   // [nblk] vector index - matrix index
    const int* blk_list = nullptr; // [nblk] gather-list block
    const int* blk_prob = nullptr; // [nblk] problem
    const int* prob_b0 = nullptr;  // [P+1] blocks of problem p: prob_b0[p] .. prob_b0[p+1]
    int maxbp = 0;                 // largest number of blocks of one problem
    const int* pflag = nullptr;    // [P] bit 0: done (skip), bit 1: finalise now
    int sms = 0;                   // SMs of the device (one-wave test of the fused step)
    unsigned long long* gsync = nullptr;  // fused step: [0], [2] grid arrival counters (reset per cycle), [1] a wait gave up
    int gwait_extra = 0;           // fused step: arrivals waited for beyond the launch's blocks (0; > 0 tests give-up)

    // sketch: the gather lists of list block L, group g of 32 sketch rows start at unit seg[L*ng + g] of ent
    // (ng = ceil(s / 32); 16-byte units, the group's lists interleaved, see common.cuh)
    int s = 0, zeta = 0, kind = 0;
    const int* seg = nullptr;
    const uint16_t* ent = nullptr;
    double sk_scale = 1.0;
    int sk_headroom = 0;  // extra right shift of the FP64 fixed-point sketch terms (long gather lists)

    // inner cycle (per-problem arrays are problem-major)
    int prec = kFP64, m = 0, t = 0;
    void* U = nullptr;         // basis storage, (m+1) vectors of N (VT); b_l = sigma[p][l] u_l for problem p
    void* W = nullptr;         // w' = A u_i (AT[N])
    double* sigma = nullptr;   // [P][m+1] 1/||u_l||
    void* normpart = nullptr;  // AT[nblk]
    void* hpart = nullptr;     // AT[nblk * kMaxTrunc]
    void* cpart = nullptr;     // AT[nblk * s]
    double* C = nullptr;       // [P][m][s]  S A b_i
    double* Q = nullptr;       // [P][m][s]  column-major: Q[l*s + r]
    double* Qt = nullptr;      // [P][s][m]  the same, row-major: Qt[r*m + l]
    double* R = nullptr;       // [P][m][m]  column-major, R[i*m + l] = R_{l,i}
    double* d = nullptr;       // [P][m]
    double* e = nullptr;       // [P][s]     running sketched residual
    double* c0 = nullptr;      // [P][s]     S v
    double* rho = nullptr;     // [P][m]
    double* y = nullptr;       // [P][m]
    double* coef = nullptr;    // [P][m]     y_l * sigma_l
    double* hco = nullptr;     // [P][m][kMaxTrunc] truncated-Arnoldi coefficients
    CycleState* cyc = nullptr; // [P]
    int qr_cluster = 8;        // CTAs per problem (one cluster) in the sketched-QR kernel; 0: the single-CTA kernel

    // outer FGMRES
    int jmax = 0;
    int outer_variant = 0;     // 0: FGMRES (least squares, Algorithm 1); 1: FFOM (square system, residual of Eq. 4)
    double* Vb = nullptr;      // [(jmax+1) * N] unnormalised outer basis, v_l = nu[p][l] Vb_l
    double* Z = nullptr;       // [jmax * N]
    double* nu = nullptr;      // [P][jmax+1]
    double* Wo = nullptr;      // [N] outer work vector
    double* opart = nullptr;   // [nblk][jmax+1]
    double* npart = nullptr;   // [nblk]
    double* npart2 = nullptr;  // [nblk]
    double* h1 = nullptr;      // [P][jmax+1]
    double* h2 = nullptr;      // [P][jmax+1]
    double* H = nullptr;       // [P][(jmax+1) * jmax] column-major, rotated in place
    double* cs = nullptr;      // [P][jmax]
    double* sn = nullptr;      // [P][jmax]
    double* g = nullptr;       // [P][jmax+1]
    double* yo = nullptr;      // [P][jmax]
    double* est_hist = nullptr;   // [P][jmax]
    double* ffom_hist = nullptr;  // [P][jmax]
    double* ires_hist = nullptr;  // [P][jmax] ||v_j - A z_j|| (true residual of inner cycle j, v_j a unit vector)
    double* rho_hist = nullptr;   // [P][jmax] the cycle's sketched residual rho_k (its estimate of that norm)
    int* k_hist = nullptr;        // [P][jmax]
    int* reason_hist = nullptr;   // [P][jmax]
    OuterState* ost = nullptr;    // [P]

    // right preconditioning (ILU(0), single FP64 system): the factors, and xin, the vector the inner SpMV multiplies
    // in place of the basis vector u_i (t_i = M^{-1} u_i); null without a preconditioner
    IluDev ilu;
    const IluHost* ilu_host = nullptr;
    const double* xin = nullptr;

    cudaStream_t st = nullptr;
};

// Block geometry on the device: block b's vector rows, column shift, gather-list block and problem.
struct BlockInfo {
    int v0, len, cs, list, prob;
};
__device__ __forceinline__ BlockInfo block_info(const Plan& p, int b) {
    BlockInfo bi;
    bi.v0 = p.blk_v0[b];
    bi.len = p.blk_len[b];
    bi.cs = p.blk_cs[b];
    bi.list = p.blk_list[b];
    bi.prob = p.blk_prob[b];
    return bi;
}

// Length-class boundaries of block b's rows for the length-binned SpMV (zero when the plan has none).
__device__ __forceinline__ void block_bins(const Plan& p, const BlockInfo& bi, int& n0, int& n01) {
    n0 = p.cls ? p.cls[2 * bi.list] : 0;
    n01 = p.cls ? p.cls[2 * bi.list + 1] : 0;
}

// ---- sketch (sketch.cu) ----
// Pattern of one system's sketch: rows[j*zeta + l], neg[j*zeta + l] for its n columns.
void launch_sketch_pattern(int n, int s, int zeta, int kind, uint64_t seed, int* rows, int8_t* neg,
                           cudaStream_t st);
// Gather lists of one system's list blocks (block k holds its columns k*Bq .. min(n, (k+1)*Bq)).  Steps:
// launch_sketch_count adds the list lengths of the system into counts[k*s + r] (zeroed by the caller); once the
// counts of every system are in place, launch_group_units turns them into the 16-byte units of every group of 32
// sketch rows (32 x the group's longest list in units of 8 entries) and launch_list_scan into group starts
// seg[0 .. nl*ng] (units); the caller reads seg[nl*ng], allocates ent (8 entries per unit), pre-fills it with the
// zero-slot offset (launch_fill_u16) and calls launch_sketch_fill per system with seg pointing at the system's first
// group.
void launch_sketch_count(int n, int s, int zeta, int Bq, const int* rows, int* counts, cudaStream_t st);
void launch_group_units(int nl, int s, const int* counts, int* units, cudaStream_t st);
void launch_list_scan(const int* counts, int* seg, int len, cudaStream_t st);
void launch_sketch_fill(int n, int s, int zeta, int Bq, const int* rows, const int8_t* neg, const int* gseg,
                        uint16_t* ent, cudaStream_t st);
void launch_fill_u16(int64_t cnt, uint16_t v, uint16_t* out, cudaStream_t st);
// Reorders the entries within every list of the nl list blocks for the shared-memory banks of the kernels that sum
// them (word = 8: the FP64 fixed-point image, 4: FP32 data); max_group = G = 128 / word times the longest list,
// padding included (above 80K entries the lists keep their fill order).  After the fill, before any use of the lists.
void launch_sketch_schedule(int nl, int s, int word, int max_group, const int* gseg, uint16_t* ent, cudaStream_t st);
// part[b*s + r] = per-block sketch sums of (scale_p * x) with scale_p = xscale[p * xstride] (1 if xscale is NULL);
// optionally stores (VT)(scale_p * x) into dst.  Skips done problems.
void launch_sketch_partials(const Plan& p, const double* x, const double* xscale, int xstride, void* dst,
                            void* part);
// out[p*s + r] = sk_scale * sum over blocks of p of part[b*s + r]; out2 (optional) gets the same values
void launch_sketch_reduce(const Plan& p, const void* part, double* out, double* out2);

// ---- inner cycle (inner.cu) ----
// resets the cycle state of every problem (j < 0: no outer solve, C3 off), u_0 = vscale_p * v, c0 = S u_0, e = c0
void launch_cycle_start(const Plan& p, int j, const double* v, const double* vscale, int vstride, int c3_on,
                        double cond_thr);
void launch_inner_spmv(const Plan& p, int i);
// The fused inner step (inner SpMV kernel and Arnoldi update in one launch with a grid-wide arrival in between) when
// the plan's row blocks fit on the GPU at once and the window is at most 4; false (nothing launched) otherwise.
bool launch_inner_step(const Plan& p, int i, bool last);
// Per-precision instances behind launch_inner_spmv, launch_inner_step and launch_inner_axpy (inner_f64.cu: FP64;
// inner_f32.cu: FP32 inner; inner_bf16.cu: BF16 basis); they launch but do not count.
void inner_spmv_f64(const Plan& p, int i);
void inner_spmv_f32(const Plan& p, int i);
void inner_spmv_bf16(const Plan& p, int i);
bool inner_step_f64(const Plan& p, int i, bool last);
bool inner_step_f32(const Plan& p, int i, bool last);
bool inner_step_bf16(const Plan& p, int i, bool last);
void inner_axpy_f64(const Plan& p, int i, bool last);
void inner_axpy_f32(const Plan& p, int i, bool last);
void inner_axpy_bf16(const Plan& p, int i, bool last);
void launch_inner_axpy(const Plan& p, int i, bool last);
// Sketches whose QR working set fits in kQrSmallElems doubles of shared memory (columns 0..m-2 of Q, the new column,
// e, two projection vectors), for at most kQrSmallProblems problems, take the single-CTA sketched QR.
constexpr int kQrSmallElems = 24576;  // 192 KB
constexpr int kQrSmallProblems = 16;
inline bool qr_small_fits(int s, int m) { return (int64_t)s * (m + 1) + 2 * (int64_t)m <= kQrSmallElems; }
cudaError_t launch_inner_qr(const Plan& p, int i, cudaStream_t st);  // on stream st (cluster or single-CTA kernel)
void launch_inner_finish(const Plan& p, double* z);  // y = R^{-1} d, z = sum_l y_l b_l (FP64)
void launch_export_basis(const Plan& p, double* out, int count);  // out[l*N + r] = sigma_l * u_l[r] (FP64)

// ---- ILU(0) right preconditioning (precond.cu) ----
// lu = the values of P A P^T (gathered from A's values), then ILU(0) colour by colour; *bad |= 1 on a zero pivot
cudaError_t launch_ilu_factor(const IluHost& H, const double* val, int* bad, cudaStream_t st);
// out = M^{-1} u = P^T (L U)^{-1} P u in the original order (u and out n float64, distinct); i >= 0: step i of the
// plan's cycle (the passes return at once once the cycle has stopped), i < 0: always
void launch_ilu_apply(const Plan& P, int i, const double* u, double* out);

// ---- outer FGMRES and helpers (outer.cu) ----
// rb = b - A x (x may be NULL = 0), npart/npart2 partials of ||rb||^2 and ||b||^2; rb may be NULL.
// only_final: restrict to problems flagged "finalise now"
void launch_residual(const Plan& p, const double* b, const double* x, double* rb, bool only_final);
void launch_init_state(const Plan& p, double tol);             // beta, ||b||, nu_0 per problem
void launch_outer_step(const Plan& p, int j);                  // w = A z_j, CGS2 against v_0..v_j, Givens update
void launch_final_x(const Plan& p, int J, const double* x0, double* x);  // problems flagged "finalise now"
void launch_true_residual_reduce(const Plan& p);               // ost[p].true_res2 from npart (flagged problems)
void launch_spmv_f64(const Plan& p, const double* x, double* y);

// ---- transpose and pattern gradient (transpose.cu) ----
// counts: int[n] zeroed by the caller; rpT int[n+1]; colT, srcT int[nnz]; maxlen int (zeroed) gets the longest row
void launch_transpose(int n, int64_t nnz, const int* rp, const int* col, int* counts, int* rpT, int* colT,
                      int* srcT, int* maxlen, cudaStream_t st);
void launch_gather_vals(int64_t nnz, const int* src, const double* val, double* out, cudaStream_t st);
void launch_pattern_outer(int n, const int* rp, const int* col, const double* u, const double* v, double alpha,
                          double* out, cudaStream_t st);
// Row order of every matrix row block (nl blocks, block L = rows lb_m0[L] .. + lb_len[L]) for the length-binned
// SpMV: perm[m0 + i] = local offset of the i-th row in (class, length, position) order; cls[2L], cls[2L+1] = number
// of rows with at most 16 and at most 64 entries.
void launch_bin_rows(int nl, const int* rp, const int* lb_m0, const int* lb_len, uint16_t* perm, int* cls,
                     cudaStream_t st);
// The length-binned SpMV's copy: lens [n] (scratch) and brp [n + 1] from the row order perm of every list block
// (launch_bcopy_build), then columns (when bcol is not null) and values in that order (launch_bcopy_fill).
void launch_bcopy_build(int n, int nl, const int* rp, const int* lb_m0, const int* lb_len, const uint16_t* perm,
                        int* lens, int* brp, cudaStream_t st);
void launch_bcopy_fill(int nl, const int* rp, const int* col, const double* val, const int* lb_m0,
                       const int* lb_len, const uint16_t* perm, const int* brp, int* bcol, double* bval,
                       cudaStream_t st);
// SELL-32 copy of a matrix whose rows have at most 255 entries: ns slices of 32 rows, slice s covering rows
// moff[q] + 32 (s - sl0[q]) .. of system q (sl0: first slice of each system, nsys + 1 entries).  launch_sell_build
// writes the row lengths len[ns * 32], the slice widths wid[ns] and their prefix sums off[ns + 1] (in units of 32
// entries); launch_sell_fill writes columns (when scol is not null) and values in slice order.
void launch_sell_build(int ns, const int* sl0, int nsys, const int* moff, const int* rp, uint8_t* len, int* wid,
                       int* off, cudaStream_t st);
void launch_sell_fill(int ns, const int* sl0, int nsys, const int* moff, const int* rp, const int* col,
                      const double* val, const int* off, const uint8_t* len, int* scol, double* sval,
                      cudaStream_t st);

// Raise the dynamic shared-memory limit of kernel `func` to at least `bytes` (cached per kernel).
void set_smem(const void* func, size_t bytes);

// launch counter (incremented by every launcher)
extern thread_local int64_t g_launches;

}  // namespace sfg
