// C ABI of the sketched-FGMRES library: handle management, validation, workspaces and the host-side driver loop.
//
// A handle holds Q >= 1 systems as one block-diagonal CSR matrix (sfgmres_create: Q = 1).  A solve with R right-hand
// sides per system runs the P = Q * R problems (system q, right-hand side r; problem p = q * R + r) in lockstep: every
// kernel covers all problems and skips the row blocks of problems that are done.  The device state
// (CycleState / OuterState per problem) carries the decisions of the stop rules, so the host synchronises once per
// outer FGMRES step to read every problem's convergence flags and to mark the problems to finalise or retire.
#include "../../include/sfgmres.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

using namespace sfg;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

// Row-block geometry of a solve with `nrhs` right-hand sides per system (device tables in one allocation).
struct Geo {
    int nrhs = -1, ver = -1;
    int P = 0, N = 0, nblk = 0;
    DevBuf tab;  // int: blk_v0, blk_len, blk_cs, blk_list, blk_prob [nblk each], prob_b0 [P+1], pflag [P]
    uint64_t used = 0;
    int maxbp = 0;           // largest number of blocks of one problem
};

constexpr int kGeoCache = 4;

}  // namespace

namespace sfg {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace sfg

struct sfgmres_ctx {
    int dev = 0;
    int nsys = 1;
    int n = 0;                  // rows of the block-diagonal matrix (sum over systems)
    int64_t nnz = 0;
    std::vector<int> sys_n;     // rows of each system
    std::vector<int> sys_moff;  // first row of each system (nsys + 1 entries)
    int* rp = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    float* val32 = nullptr;
    // transpose (built on first use): row pointers, columns, source positions in A, values, FP32 values
    int* rpT = nullptr;
    int* colT = nullptr;
    int* srcT = nullptr;
    double* valT = nullptr;
    float* val32T = nullptr;
    int maxlenT = 0, vecT = 8;
    // SELL-32 copies of A ([0]) and A^T ([1]) for the one-thread-per-row FP64 inner SpMV, built on first use
    struct Sell {
        int* off = nullptr;
        uint8_t* len = nullptr;
        int* col = nullptr;
        double* val = nullptr;
        int64_t total = 0;  // entries, padding included
    } sell[2];
    int sl_ns = 0;                 // slices (the same for A and A^T: block-diagonal with the same blocks)
    int* sl_sys = nullptr;         // [nsys + 1] first slice of each system, then [nsys + 1] first row of each system
    int* sl_base = nullptr;        // [list blocks] first slice of each list block
    int sl_base_ver = -1;
    uint64_t seed = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t qst = nullptr;       // side stream of the sketched-QR kernel
    cudaEvent_t ev_c = nullptr;       // "sketched column ready" (main -> side)
    cudaEvent_t ev_q = nullptr;       // "cycle's QR updates done" (side -> main)
    int sms = 152;
    int maxlen = 0;                   // longest CSR row

    // options
    int prec = kFP64, zeta = 8, c3 = 1, max_outer = 50, kind = 0, profile = 0, vec_opt = 0, block_rows = 0;
    int use_graph = 1;
    int fuse_step = 1;  // 1: one launch per inner step where the row blocks fit on the GPU at once
    int outer_variant = 0;  // 0: FGMRES; 1: FFOM
    int precond = 0;        // 0: none; 1: ILU(0) in a multicolour order, right preconditioning
    int wait_extra = 0;  // fused step: arrivals waited for beyond the launch's blocks (test of the give-up path)
    bool step_fused = false;  // the last cycle ran the fused inner step
    double cond_thr = 1e15;

    // list-block geometry (depends on the systems and the block-rows option; version bumps on change)
    int Bn = 0, vec = 8, nl = 0, geo_ver = 0;
    std::vector<int> sys_Bq, sys_l0;

    // vector-block geometries, cached per number of right-hand sides
    Geo geos[kGeoCache];
    uint64_t geo_clock = 0;

    // length-binned SpMV row orders for A [0] and A^T [1] (built for one geometry version), and the matrix row
    // blocks' first rows and lengths on the device
    uint16_t* perm[2] = {nullptr, nullptr};
    int* cls[2] = {nullptr, nullptr};
    int bins_ver[2] = {-1, -1};
    int* lb = nullptr;  // lb_m0 [nl], lb_len [nl]
    int lb_ver = -1;
    // the length-binned SpMV's FP64 copies of A [0] and A^T [1] with each row block's rows in its processing order
    // (built for one geometry version; values follow sfgmres_update_values)
    struct BCopy {
        int* rp = nullptr;
        int* col = nullptr;
        double* val = nullptr;
        int ver = -1;
    } bc[2];

    // sketch gather lists (cached for one (s, zeta, kind, geometry version))
    int sk_s = -1, sk_zeta = -1, sk_kind = -1, sk_ver = -1, sk_headroom = 0, sk_word = 0;
    int* seg = nullptr;
    uint16_t* ent = nullptr;

    // workspaces
    DevBuf U, W, sigma, normpart, hpart, cpart, C, Q, Qt, R, d, e, c0, rho, y, coef, hco, cyc;
    DevBuf Vb, Z, nu, Wo, opart, npart, npart2, h1, h2, H, cs, sn, g, yo, est_hist, ffom_hist, ires_hist, rho_hist,
        k_hist, reason_hist,
        ost;
    DevBuf bst, xst, x0st;  // staging / internal copies
    // ILU(0) right preconditioner (built on first use; the factors follow sfgmres_update_values)
    IluHost ilu;
    std::vector<int> ilu_colour;  // colour of every row (original order)
    std::vector<int> ilu_src;     // host copy of ilu.src
    DevBuf ilu_rp, ilu_col, ilu_diag, ilu_perm, ilu_src_d, ilu_lu, ilu_y, ilu_zp, ilu_t, ilu_zt, ilu_bad;
    int ilu_built = 0;            // structure built
    int ilu_vals_ver = -1;        // values version the factors were computed for
    int vals_ver = 0;             // bumped by sfgmres_update_values
    // outer workspaces of the lower levels of sfgmres_solve_multilevel (level 1, 2, ...)
    struct LevelWs {
        DevBuf Vb, Z, nu, Wo, opart, npart, npart2, h1, h2, H, cs, sn, g, yo, est_hist, ffom_hist, ires_hist,
            rho_hist, k_hist, reason_hist, ost, pflag, rhs;
    };
    std::vector<LevelWs> lvl;
    DevBuf gsync;           // fused inner step: grid arrival counters [0], [2] and give-up flag [1] (u64)

    // pinned host mirrors of the per-problem device state
    HostBuf h_ost, h_cyc, h_pflag;

    // executable graphs of outer steps j = 0, 1, ... (one inner cycle + one outer FGMRES step each), valid for the
    // plan they were captured with
    std::vector<uint64_t> graph_key;
    std::vector<cudaGraphExec_t> graph_exec;
    std::vector<int64_t> graph_launches;

    // profiling: event pairs per inner kernel; outer step j records its m launches of each kernel into pairs
    // [base, base + m) of each pool (captured into the step's graph, or recorded as the kernels are launched)
    std::vector<EventPair> ev_spmv, ev_axpy, ev_qr;
    size_t ev_next = 0;   // next free pair (the same index in all three pools)
    size_t ev_graph = 0;  // pairs [0, ev_graph) belong to the cached graphs
    std::vector<size_t> graph_ev;           // base pair of each cached graph (SIZE_MAX: captured without events)
    std::vector<std::pair<int, size_t>> ev_steps;  // this solve's outer steps: (j, base pair)
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;

    std::string err;
};

namespace {

int fail(sfgmres_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e__ = (call);                                                                         \
        if (e__ != cudaSuccess)                                                                           \
            return fail(h, e__ == cudaErrorMemoryAllocation ? SFGMRES_ERR_OOM : SFGMRES_ERR_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e__));                             \
    } while (0)

int ensure(sfgmres_ctx* h, DevBuf& b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    if (b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(h, SFGMRES_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    b.bytes = bytes;
    return 0;
}

int ensure_host(sfgmres_ctx* h, HostBuf& b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    if (b.bytes >= bytes) return 0;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMallocHost(&b.p, bytes) != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(h, SFGMRES_ERR_OOM, "cudaMallocHost of " + std::to_string(bytes) + " bytes failed");
    }
    b.bytes = bytes;
    return 0;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void release_host(HostBuf& b) {
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// SpMV shape: one thread per row when every row is short (stencils), else the length-binned SpMV (0).
int choose_vec(int64_t, int, int maxlen) { return maxlen <= 16 ? 1 : 0; }

// Row blocks of one system: nblk a multiple of the SM count where possible, Bn a multiple of 32, <= kBlockRowsMax.
// FP64 inner cycles size the blocks for all SMs but one QR cluster's: the sketched QR of step i runs beside the
// fused inner kernel of step i+1, and a one-wave FP64 inner kernel whose CTAs share SMs with the QR cluster waits
// on those stragglers (measured on 128^3: 137 us per step with 304 blocks, 112 us with 288).  The FP32 and BF16
// inner kernels are short enough that the QR does not slow them, and all SMs serve them best.
int single_block_rows(int n, int sms, int prec) {
    if (prec == 0 && sms > 2 * kQrCluster) sms -= kQrCluster;
    int q = 1, b = 32;
    for (;;) {
        const int64_t per = ((int64_t)n + (int64_t)sms * q - 1) / ((int64_t)sms * q);
        b = (int)(((per + 31) / 32) * 32);
        if (b <= kBlockRowsMax) break;
        q *= 2;
    }
    return std::max(b, 32);
}

// Rows per block of a batch of systems (every system is cut into blocks of this size; the last block of a system
// is ragged).  4096 rows = 8 rows per thread of a 512-thread CTA: enough independent rows per thread to hide the
// gather latency, and the shared-memory block (32 KiB in FP64) leaves room for two CTAs per SM.
constexpr int kBatchBlockRows = 4096;

void set_list_geometry(sfgmres_ctx* h) {
    h->sys_Bq.assign(h->nsys, 0);
    h->sys_l0.assign(h->nsys + 1, 0);
    int Bq;
    if (h->block_rows) Bq = h->block_rows;
    else if (h->nsys == 1) Bq = single_block_rows(h->n, h->sms, h->prec);
    else Bq = kBatchBlockRows;
    int Bn = 32, nl = 0;
    for (int q = 0; q < h->nsys; ++q) {
        const int nq = h->sys_n[q];
        h->sys_Bq[q] = Bq;
        h->sys_l0[q] = nl;
        nl += (nq + Bq - 1) / Bq;
        Bn = std::max(Bn, std::min(Bq, ((nq + 31) / 32) * 32));
    }
    h->sys_l0[h->nsys] = nl;
    h->nl = nl;
    h->Bn = Bn;
    ++h->geo_ver;
}

// CTAs per problem of the sketched-QR update.  Small sketches of few problems whose inner step leaves an SM with at
// most one of its CTAs (nblk <= sms): 0, the single-CTA kernel (512 threads; its reductions cost shared-memory
// barriers instead of cluster barriers and distributed-shared-memory exchanges).  It needs a large share of an SM's
// registers and shared memory, so beside an inner step that fills every SM it would wait for the step to end (the
// random Zipf workload, s = 240: 335 -> 361 ms per FP64 solve).  Otherwise a cluster of small CTAs (they fit beside
// the step's) with as many CTAs as the batch leaves room for: the update is bound by the latency of its reads, which
// more SMs hide better.
int qr_cluster_for(int P, int s, int m, int nblk, int sms) {
    if (P <= kQrSmallProblems && qr_small_fits(s, m) && nblk <= sms) return 0;  // one CTA per problem
    if (P <= 16) return kQrCluster;
    if (P <= 32) return 4;
    if (P <= 64) return 2;
    return 1;
}

// ---- CSR validation on the device ----
// bad[0] |= 1 range, 2 row_ptr[0] != 0, 4 row_ptr[n] != nnz, 8 decreasing, 16 column out of range, 32 column
// outside the row's system; bad[1] = longest row.
__global__ void k_validate_csr(int n, int64_t nnz, const int64_t* __restrict__ rp64, const int* __restrict__ col,
                               int* __restrict__ rp32, int* __restrict__ bad, const int* __restrict__ moff,
                               int nsys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) {
        const int64_t v = rp64[i];
        if (v < 0 || v > nnz) atomicOr(bad, 1);
        if (i == 0 && v != 0) atomicOr(bad, 2);
        if (i == n && v != nnz) atomicOr(bad, 4);
        if (i < n && rp64[i + 1] < v) atomicOr(bad, 8);
        if (i < n) {
            const int64_t e = rp64[i + 1];
            const int64_t len = e - v;
            if (len > 0) atomicMax(bad + 1, (int)min(len, (int64_t)INT32_MAX));
            if (nsys > 1 && v >= 0 && e <= nnz && v <= e) {
                int lo = 0, hi = nsys;  // system of row i: moff[lo] <= i < moff[lo + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (moff[mid] <= i) lo = mid;
                    else hi = mid;
                }
                const int c0 = moff[lo], c1 = moff[lo + 1];
                for (int64_t q = v; q < e; ++q) {
                    const int c = col[q];
                    if (c < c0 || c >= c1) {
                        atomicOr(bad, 32);
                        break;
                    }
                }
            }
        }
        rp32[i] = (int)v;
    }
    if (i < nnz) {
        const int c = col[i];
        if (c < 0 || c >= n) atomicOr(bad, 16);
    }
}

__global__ void k_to_f32(int64_t nnz, const double* __restrict__ v, float* __restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)v[i];
}

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = v;
}

// x += a z
__global__ void k_axpy_scalar(int64_t n, double a, const double* __restrict__ z, double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += a * z[i];
}

// x = 0 over the rows of the problems whose flag has bit 2 set (right-hand side zero).
// b = scale[0] * v (the right-hand side of a lower level of the multi-level FGMRES: the parent's outer vector v_j,
// stored unnormalised with its scale nu_j on the device)
__global__ void k_scale_copy(int64_t n, const double* __restrict__ v, const double* __restrict__ scale,
                             double* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = scale[0] * v[i];
}

// The cycle-state fields the outer Givens kernel records, set from a completed lower-level FGMRES run (the multi-level
// FGMRES's preconditioner): its outer steps, why it stopped (3 met its tolerance, 1 budget), its last estimate.
__global__ void k_set_cycle(CycleState* cyc, int k, int reason, double rho) {
    cyc->k = k;
    cyc->reason = reason;
    cyc->rho = rho;
    cyc->stopped = 1;
}

__global__ void k_zero_flagged(const Plan P, double* __restrict__ x) {
    const BlockInfo bi = block_info(P, blockIdx.x);
    if (!(P.pflag[bi.prob] & 4)) return;
    for (int k = threadIdx.x; k < bi.len; k += blockDim.x) x[bi.v0 + k] = 0.0;
}

__global__ void k_neg_to_sign(int64_t cnt, const int8_t* __restrict__ a, int8_t* __restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = a[i] ? (int8_t)-1 : (int8_t)1;
}

int grid_for(int64_t n, int th = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + th - 1) / th, 152 * 16)); }

// Gather lists of every system's sketch for s rows (one pattern per system, all drawn from the handle's seed).
int build_sketch(sfgmres_ctx* h, int s) {
    const int zeta = (h->kind == 1) ? 1 : h->zeta;
    const int word = (h->prec == kFP64) ? 8 : 4;  // the summed words: FP64 fixed-point image, or FP32 data
    if (h->seg && h->sk_s == s && h->sk_zeta == zeta && h->sk_kind == h->kind && h->sk_ver == h->geo_ver &&
        h->sk_word == word)
        return 0;
    if (h->seg) cudaFree(h->seg);
    if (h->ent) cudaFree(h->ent);
    h->seg = nullptr;
    h->ent = nullptr;
    h->sk_s = -1;
    int maxn = 0;
    for (int q = 0; q < h->nsys; ++q) maxn = std::max(maxn, h->sys_n[q]);
    const int ng = (s + 31) / 32;  // groups of 32 sketch rows per list block
    const int64_t ncnt = (int64_t)h->nl * s;
    const int64_t nseg = (int64_t)h->nl * ng + 1;
    if (ncnt >= INT32_MAX || nseg >= INT32_MAX)
        return fail(h, SFGMRES_ERR_INVALID_ARG, "sketch too large for 32-bit gather lists");
    int* rows = nullptr;
    int8_t* neg = nullptr;
    int* counts = nullptr;
    int* units = nullptr;
    const int64_t tq = (int64_t)maxn * zeta;
    CK(cudaMalloc(&rows, tq * sizeof(int)));
    CK(cudaMalloc(&neg, tq));
    CK(cudaMalloc(&counts, ncnt * sizeof(int)));
    CK(cudaMalloc(&units, nseg * sizeof(int)));
    CK(cudaMalloc(&h->seg, nseg * sizeof(int)));
    CK(cudaMemsetAsync(counts, 0, ncnt * sizeof(int), h->st));
    for (int q = 0; q < h->nsys; ++q) {
        launch_sketch_pattern(h->sys_n[q], s, zeta, h->kind, h->seed, rows, neg, h->st);
        launch_sketch_count(h->sys_n[q], s, zeta, h->sys_Bq[q], rows, counts + (int64_t)h->sys_l0[q] * s, h->st);
    }
    launch_group_units(h->nl, s, counts, units, h->st);
    launch_list_scan(units, h->seg, (int)(nseg - 1), h->st);
    std::vector<int> hs(nseg);
    CK(cudaMemcpyAsync(hs.data(), h->seg, nseg * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const int64_t total = (int64_t)hs[nseg - 1] * 8;  // entries
    if (hs[nseg - 1] < 0 || total >= ((int64_t)1 << 34))
        return fail(h, SFGMRES_ERR_INVALID_ARG, "sketch too large for 32-bit gather lists");
    CK(cudaMalloc(&h->ent, std::max<int64_t>(total, 8) * sizeof(uint16_t)));
    launch_fill_u16(total, (uint16_t)h->Bn, h->ent, h->st);  // padding points at the zero slot
    for (int q = 0; q < h->nsys; ++q) {
        launch_sketch_pattern(h->sys_n[q], s, zeta, h->kind, h->seed, rows, neg, h->st);
        launch_sketch_fill(h->sys_n[q], s, zeta, h->sys_Bq[q], rows, neg, h->seg + (int64_t)h->sys_l0[q] * ng,
                           h->ent, h->st);
    }
    // the longest list (padding included), in entries: E * 8 for the group with the most units
    int longest = 0;
    for (int64_t q = 0; q + 1 < nseg; ++q) longest = std::max(longest, (hs[q + 1] - hs[q]) / 32 * 8);
    launch_sketch_schedule(h->nl, s, word, (128 / word) * longest, h->seg, h->ent, h->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    cudaFree(rows);
    cudaFree(neg);
    cudaFree(counts);
    cudaFree(units);
    {
        // FP64 sketch terms are 53-bit integers summed exactly in 64 bits: lists longer than 1023 entries get
        // extra right shifts so that no sum can overflow (padding entries add zero)
        int H = 0;
        while ((longest >> H) >= 1023) ++H;
        h->sk_headroom = H;
    }
    h->sk_s = s;
    h->sk_zeta = zeta;
    h->sk_kind = h->kind;
    h->sk_word = word;
    h->sk_ver = h->geo_ver;
    return 0;
}

// Vector-block geometry for nrhs right-hand sides per system (cached; the least recently used entry is replaced).
int get_geometry(sfgmres_ctx* h, int nrhs, Geo** out) {
    Geo* g = nullptr;
    for (Geo& c : h->geos)
        if (c.nrhs == nrhs && c.ver == h->geo_ver) g = &c;
    if (!g) {
        const int64_t N64 = (int64_t)nrhs * h->n;
        if (N64 > INT32_MAX - 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "nrhs * n must be below 2^31 - 1");
        g = &h->geos[0];
        for (Geo& c : h->geos)
            if (c.used < g->used) g = &c;
        const int P = h->nsys * nrhs;
        std::vector<int> v0, len, cs, lst, prob, pb0(P + 1);
        for (int q = 0; q < h->nsys; ++q) {
            const int nq = h->sys_n[q], Bq = h->sys_Bq[q], mo = h->sys_moff[q];
            const int nlq = (nq + Bq - 1) / Bq;
            for (int r = 0; r < nrhs; ++r) {
                const int p = q * nrhs + r;
                const int pv0 = nrhs * mo + r * nq;
                pb0[p] = (int)v0.size();
                for (int k = 0; k < nlq; ++k) {
                    v0.push_back(pv0 + k * Bq);
                    len.push_back(std::min(Bq, nq - k * Bq));
                    cs.push_back(pv0 - mo);
                    lst.push_back(h->sys_l0[q] + k);
                    prob.push_back(p);
                }
            }
        }
        const int nblk = (int)v0.size();
        pb0[P] = nblk;
        std::vector<int> tab;
        tab.reserve((size_t)5 * nblk + 2 * P + 1);
        for (auto* vv : {&v0, &len, &cs, &lst, &prob}) tab.insert(tab.end(), vv->begin(), vv->end());
        tab.insert(tab.end(), pb0.begin(), pb0.end());
        tab.resize(tab.size() + P, 0);  // pflag
        g->nrhs = -1;
        int rc = ensure(h, g->tab, tab.size() * sizeof(int));
        if (rc) return rc;
        CK(cudaMemcpyAsync(g->tab.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
        CK(cudaStreamSynchronize(h->st));
        g->nrhs = nrhs;
        g->ver = h->geo_ver;
        g->maxbp = 0;
        for (int p = 0; p < P; ++p) g->maxbp = std::max(g->maxbp, pb0[p + 1] - pb0[p]);
        g->P = P;
        g->N = (int)N64;
        g->nblk = nblk;
    }
    g->used = ++h->geo_clock;
    *out = g;
    return 0;
}

int ensure_f32(sfgmres_ctx* h, bool transpose) {
    float*& v32 = transpose ? h->val32T : h->val32;
    if (v32) return 0;
    CK(cudaMalloc(&v32, std::max<int64_t>(h->nnz, 1) * sizeof(float)));
    k_to_f32<<<grid_for(h->nnz), 256, 0, h->st>>>(h->nnz, transpose ? h->valT : h->val, v32);
    CK(cudaGetLastError());
    return 0;
}

// A^T in CSR form, built on first use (deterministic layout) and kept; values follow sfgmres_update_values.  The
// transpose of the block-diagonal matrix is block-diagonal with the same blocks, so the row-block geometry and the
// sketch lists serve both.
int ensure_transpose(sfgmres_ctx* h) {
    if (h->rpT) return 0;
    const int64_t nz = std::max<int64_t>(h->nnz, 1);
    int* counts = nullptr;
    int* mx = nullptr;
    CK(cudaMalloc(&h->rpT, ((size_t)h->n + 1) * sizeof(int)));
    CK(cudaMalloc(&h->colT, nz * sizeof(int)));
    CK(cudaMalloc(&h->srcT, nz * sizeof(int)));
    CK(cudaMalloc(&h->valT, nz * sizeof(double)));
    CK(cudaMalloc(&counts, (size_t)h->n * sizeof(int)));
    CK(cudaMalloc(&mx, sizeof(int)));
    CK(cudaMemsetAsync(counts, 0, (size_t)h->n * sizeof(int), h->st));
    CK(cudaMemsetAsync(mx, 0, sizeof(int), h->st));
    launch_transpose(h->n, h->nnz, h->rp, h->col, counts, h->rpT, h->colT, h->srcT, mx, h->st);
    launch_gather_vals(h->nnz, h->srcT, h->val, h->valT, h->st);
    CK(cudaMemcpyAsync(&h->maxlenT, mx, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    cudaFree(counts);
    cudaFree(mx);
    h->vecT = choose_vec(h->nnz, h->n, h->maxlenT);
    return 0;
}

// Row orders of the length-binned SpMV for A (or A^T), built for the current row-block geometry.
int ensure_bins(sfgmres_ctx* h, bool transpose) {
    const int t = transpose ? 1 : 0;
    if (h->bins_ver[t] == h->geo_ver && h->perm[t]) return 0;
    if (h->lb_ver != h->geo_ver) {
        if (h->lb) cudaFree(h->lb);
        h->lb = nullptr;
        std::vector<int> hb(2 * (size_t)h->nl);
        for (int q = 0; q < h->nsys; ++q) {
            const int nq = h->sys_n[q], Bq = h->sys_Bq[q];
            for (int k = 0, L = h->sys_l0[q]; k * Bq < nq; ++k, ++L) {
                hb[L] = h->sys_moff[q] + k * Bq;
                hb[h->nl + L] = std::min(Bq, nq - k * Bq);
            }
        }
        CK(cudaMalloc(&h->lb, hb.size() * sizeof(int)));
        CK(cudaMemcpy(h->lb, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice));
        h->lb_ver = h->geo_ver;
    }
    if (!h->perm[t]) CK(cudaMalloc(&h->perm[t], std::max<size_t>(h->n, 1) * sizeof(uint16_t)));
    if (h->cls[t]) cudaFree(h->cls[t]);
    h->cls[t] = nullptr;
    CK(cudaMalloc(&h->cls[t], 2 * (size_t)h->nl * sizeof(int)));
    launch_bin_rows(h->nl, transpose ? h->rpT : h->rp, h->lb, h->lb + h->nl, h->perm[t], h->cls[t], h->st);
    CK(cudaGetLastError());
    h->bins_ver[t] = h->geo_ver;
    return 0;
}

// The length-binned SpMV's copy of A (or A^T): every row block's rows stored in the order the SpMV processes them
// (the bins of the current geometry), FP64 values.
int ensure_bcopy(sfgmres_ctx* h, bool transpose) {
    const int t = transpose ? 1 : 0;
    sfgmres_ctx::BCopy& B = h->bc[t];
    if (B.ver == h->geo_ver && B.rp) return 0;
    const int* rp = transpose ? h->rpT : h->rp;
    const int* col = transpose ? h->colT : h->col;
    const double* val = transpose ? h->valT : h->val;
    const size_t n = (size_t)h->n, nnz = (size_t)std::max<int64_t>(h->nnz, 1);
    if (!B.rp) {
        CK(cudaMalloc(&B.rp, (n + 1) * sizeof(int)));
        CK(cudaMalloc(&B.col, nnz * sizeof(int)));
        CK(cudaMalloc(&B.val, nnz * sizeof(double)));
    }
    int* lens = nullptr;
    CK(cudaMalloc(&lens, std::max<size_t>(n, 1) * sizeof(int)));
    launch_bcopy_build(h->n, h->nl, rp, h->lb, h->lb + h->nl, h->perm[t], lens, B.rp, h->st);
    launch_bcopy_fill(h->nl, rp, col, val, h->lb, h->lb + h->nl, h->perm[t], B.rp, B.col, B.val, h->st);
    CK(cudaStreamSynchronize(h->st));
    cudaFree(lens);
    CK(cudaGetLastError());
    B.ver = h->geo_ver;
    return 0;
}

// SELL-32 copy of A (or A^T) for the one-thread-per-row FP64 inner SpMV (measured faster there; the FP32 inner
// kernel keeps the CSR arrays, which measured as fast or faster); the list blocks' first slices follow the
// row-block geometry.
int ensure_sell(sfgmres_ctx* h, bool transpose) {
    sfgmres_ctx::Sell& S = h->sell[transpose ? 1 : 0];
    const int* rp = transpose ? h->rpT : h->rp;
    const int* col = transpose ? h->colT : h->col;
    const double* val = transpose ? h->valT : h->val;
    if (!h->sl_sys) {
        std::vector<int> t(2 * (size_t)(h->nsys + 1), 0);
        int64_t ns = 0;
        for (int q = 0; q < h->nsys; ++q) {
            t[q] = (int)ns;
            ns += (h->sys_n[q] + 31) / 32;
        }
        if (ns > INT32_MAX - 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "too many rows for the SELL-32 layout");
        t[h->nsys] = (int)ns;
        for (int q = 0; q <= h->nsys; ++q) t[h->nsys + 1 + q] = h->sys_moff[q];
        CK(cudaMalloc(&h->sl_sys, t.size() * sizeof(int)));
        CK(cudaMemcpy(h->sl_sys, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice));
        h->sl_ns = (int)ns;
    }
    const int ns = h->sl_ns;
    const int* sl0 = h->sl_sys;
    const int* moff = h->sl_sys + h->nsys + 1;
    if (!S.off) {
        int* wid = nullptr;
        CK(cudaMalloc(&S.off, ((size_t)ns + 1) * sizeof(int)));
        CK(cudaMalloc(&S.len, std::max<size_t>((size_t)ns * 32, 1)));
        CK(cudaMalloc(&wid, std::max<size_t>((size_t)ns, 1) * sizeof(int)));
        launch_sell_build(ns, sl0, h->nsys, moff, rp, S.len, wid, S.off, h->st);
        int tot = 0;
        CK(cudaMemcpyAsync(&tot, S.off + ns, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        cudaFree(wid);
        CK(cudaGetLastError());
        S.total = (int64_t)tot * 32;
        CK(cudaMalloc(&S.col, std::max<int64_t>(S.total, 1) * sizeof(int)));
        CK(cudaMalloc(&S.val, std::max<int64_t>(S.total, 1) * sizeof(double)));
        launch_sell_fill(ns, sl0, h->nsys, moff, rp, col, val, S.off, S.len, S.col, S.val, h->st);
        CK(cudaGetLastError());
    }
    if (h->sl_base_ver != h->geo_ver) {
        std::vector<int> hb((size_t)std::max(h->nl, 1), 0);
        int ns0 = 0;
        for (int q = 0; q < h->nsys; ++q) {
            const int nq = h->sys_n[q], Bq = h->sys_Bq[q];
            for (int k = 0, L = h->sys_l0[q]; k * Bq < nq; ++k, ++L) hb[L] = ns0 + k * (Bq / 32);
            ns0 += (nq + 31) / 32;
        }
        if (h->sl_base) cudaFree(h->sl_base);
        h->sl_base = nullptr;
        CK(cudaMalloc(&h->sl_base, hb.size() * sizeof(int)));
        CK(cudaMemcpy(h->sl_base, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice));
        h->sl_base_ver = h->geo_ver;
    }
    return 0;
}

// Matrix and geometry fields of a Plan (enough for the SpMV and the per-block helpers).
void plan_geometry(sfgmres_ctx* h, const Geo* g, bool transpose, Plan& P) {
    P.nnz = h->nnz;
    P.rp = transpose ? h->rpT : h->rp;
    P.col = transpose ? h->colT : h->col;
    P.val = transpose ? h->valT : h->val;
    P.val32 = transpose ? h->val32T : h->val32;
    P.vec = transpose ? (h->vec_opt ? h->vec_opt : h->vecT) : h->vec;
    P.perm = (P.vec == 0) ? h->perm[transpose ? 1 : 0] : nullptr;
    P.cls = (P.vec == 0) ? h->cls[transpose ? 1 : 0] : nullptr;
    const sfgmres_ctx::BCopy& B = h->bc[transpose ? 1 : 0];
    const bool bc = (P.vec == 0) && B.rp && B.ver == h->geo_ver && h->bins_ver[transpose ? 1 : 0] == h->geo_ver;
    P.brp = bc ? B.rp : nullptr;
    P.bcol = bc ? B.col : nullptr;
    P.bval = bc ? B.val : nullptr;
    const sfgmres_ctx::Sell& S = h->sell[transpose ? 1 : 0];
    const bool sl = (P.vec == 1) && h->prec == kFP64 && S.off && h->sl_base_ver == h->geo_ver;
    P.sl_off = sl ? S.off : nullptr;
    P.sl_len = sl ? S.len : nullptr;
    P.sl_col = sl ? S.col : nullptr;
    P.sl_val = sl ? S.val : nullptr;
    P.sl_base = sl ? h->sl_base : nullptr;
    P.N = g->N;
    P.P = g->P;
    P.nblk = g->nblk;
    P.Bn = h->Bn;
    const int* t = (const int*)g->tab.p;
    const int nb = g->nblk;
    P.blk_v0 = t;
    P.blk_len = t + nb;
    P.blk_cs = t + 2 * (int64_t)nb;
    P.blk_list = t + 3 * (int64_t)nb;
    P.blk_prob = t + 4 * (int64_t)nb;
    P.prob_b0 = t + 5 * (int64_t)nb;
    P.maxbp = g->maxbp;
    P.pflag = t + 5 * (int64_t)nb + g->P + 1;
    P.st = h->st;
}

int* pflag_of(const Geo* g) { return (int*)g->tab.p + 5 * (int64_t)g->nblk + g->P + 1; }

// Allocates the workspaces of a solve with nrhs right-hand sides per system and fills a Plan (for A, or for A^T
// when transpose is set).  Every problem's flag is reset to "active".
// ---- ILU(0) right preconditioner (set-up; the kernels are in precond.cu) ----
// Structure, once per handle: a greedy colouring of the pattern of A + A^T in the natural row order (each row takes the
// smallest colour no earlier coupled row has), the rows ordered colour by colour (natural order within a colour), and
// P A P^T in CSR with sorted columns, its diagonal positions and the source position of every entry.  This is graph
// analysis of the sparsity pattern, done on the host from a copy of the CSR structure.  Values, at every change of A's
// values: the ILU(0) factorisation on the device, one pass per colour.
int ensure_ilu(sfgmres_ctx* h) {
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "ILU(0) preconditioning needs a single-system handle");
    const int n = h->n;
    const int64_t nnz = h->nnz;
    int rc;
    if (!h->ilu_built) {
        std::vector<int> rp(n + 1), col(std::max<int64_t>(nnz, 1));
        CK(cudaMemcpy(rp.data(), h->rp, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
        if (nnz) CK(cudaMemcpy(col.data(), h->col, nnz * sizeof(int), cudaMemcpyDeviceToHost));
        // the columns' rows (the pattern of A^T) by a counting sort
        std::vector<int> tp(n + 1, 0), trow(std::max<int64_t>(nnz, 1));
        for (int64_t p = 0; p < nnz; ++p) ++tp[col[p] + 1];
        for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
        {
            std::vector<int> fill(tp.begin(), tp.end() - 1);
            for (int i = 0; i < n; ++i)
                for (int p = rp[i]; p < rp[i + 1]; ++p) trow[fill[col[p]]++] = i;
        }
        // greedy colouring in the natural order
        std::vector<int> colour(n, -1), seen;  // seen[c] == i: colour c is taken by a coupled earlier row of row i
        int ncol = 0;
        for (int i = 0; i < n; ++i) {
            auto mark = [&](int j) {
                if (j < i && colour[j] >= 0) {
                    if ((int)seen.size() <= colour[j]) seen.resize(colour[j] + 1, -1);
                    seen[colour[j]] = i;
                }
            };
            for (int p = rp[i]; p < rp[i + 1]; ++p) mark(col[p]);
            for (int p = tp[i]; p < tp[i + 1]; ++p) mark(trow[p]);
            int c = 0;
            while (c < (int)seen.size() && seen[c] == i) ++c;
            colour[i] = c;
            ncol = std::max(ncol, c + 1);
        }
        // rows colour by colour
        std::vector<int> starts(ncol + 1, 0), perm(n), inv(n);
        for (int i = 0; i < n; ++i) ++starts[colour[i] + 1];
        for (int c = 0; c < ncol; ++c) starts[c + 1] += starts[c];
        {
            std::vector<int> fill(starts.begin(), starts.end() - 1);
            for (int i = 0; i < n; ++i) perm[fill[colour[i]]++] = i;
        }
        for (int r = 0; r < n; ++r) inv[perm[r]] = r;
        // P A P^T with sorted columns, diagonal positions, source positions
        std::vector<int> prp(n + 1, 0), pcol(std::max<int64_t>(nnz, 1)), psrc(std::max<int64_t>(nnz, 1)), pdiag(n, -1);
        std::vector<std::pair<int, int>> row;
        for (int r = 0; r < n; ++r) {
            const int i = perm[r];
            row.clear();
            for (int p = rp[i]; p < rp[i + 1]; ++p) row.push_back({inv[col[p]], p});
            std::sort(row.begin(), row.end());
            prp[r + 1] = prp[r] + (int)row.size();
            for (size_t q = 0; q < row.size(); ++q) {
                if (q > 0 && row[q].first == row[q - 1].first)
                    return fail(h, SFGMRES_ERR_INVALID_ARG, "ILU(0) needs a CSR without repeated entries");
                pcol[prp[r] + q] = row[q].first;
                psrc[prp[r] + q] = row[q].second;
                if (row[q].first == r) pdiag[r] = prp[r] + (int)q;
            }
            if (pdiag[r] < 0) return fail(h, SFGMRES_ERR_INVALID_ARG, "ILU(0) needs every diagonal entry of A stored");
        }
        const size_t N = (size_t)n, Z = (size_t)std::max<int64_t>(nnz, 1);
        if ((rc = ensure(h, h->ilu_rp, (N + 1) * 4)) || (rc = ensure(h, h->ilu_col, Z * 4)) ||
            (rc = ensure(h, h->ilu_diag, N * 4)) || (rc = ensure(h, h->ilu_perm, N * 4)) ||
            (rc = ensure(h, h->ilu_src_d, Z * 4)) || (rc = ensure(h, h->ilu_lu, Z * 8)) ||
            (rc = ensure(h, h->ilu_y, N * 8)) || (rc = ensure(h, h->ilu_zp, N * 8)) ||
            (rc = ensure(h, h->ilu_t, N * 8)) || (rc = ensure(h, h->ilu_zt, N * 8)) ||
            (rc = ensure(h, h->ilu_bad, sizeof(int))))
            return rc;
        CK(cudaMemcpy(h->ilu_rp.p, prp.data(), (N + 1) * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ilu_col.p, pcol.data(), Z * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ilu_diag.p, pdiag.data(), N * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ilu_perm.p, perm.data(), N * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ilu_src_d.p, psrc.data(), Z * 4, cudaMemcpyHostToDevice));
        IluHost& H = h->ilu;
        H.n = n;
        H.ncol = ncol;
        H.nnz = nnz;
        H.starts = starts;
        H.src = (const int*)h->ilu_src_d.p;
        H.dev.rp = (const int*)h->ilu_rp.p;
        H.dev.col = (const int*)h->ilu_col.p;
        H.dev.diag = (const int*)h->ilu_diag.p;
        H.dev.perm = (const int*)h->ilu_perm.p;
        H.dev.lu = (double*)h->ilu_lu.p;
        H.dev.y = (double*)h->ilu_y.p;
        H.dev.zp = (double*)h->ilu_zp.p;
        h->ilu_colour = colour;
        h->ilu_src = psrc;
        h->ilu_built = 1;
        h->ilu_vals_ver = -1;
    }
    if (h->ilu_vals_ver != h->vals_ver) {
        CK(cudaMemsetAsync(h->ilu_bad.p, 0, sizeof(int), h->st));
        CK(launch_ilu_factor(h->ilu, h->val, (int*)h->ilu_bad.p, h->st));
        int bad = 0;
        CK(cudaMemcpyAsync(&bad, h->ilu_bad.p, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (bad) return fail(h, SFGMRES_ERR_INVALID_ARG, "ILU(0) met a zero pivot");
        h->ilu_vals_ver = h->vals_ver;
    }
    return 0;
}

int prepare(sfgmres_ctx* h, int nrhs, int m, int s, int t, int jmax, Plan* p, Geo** geo_out, bool transpose = false) {
    int rc;
    Geo* g = nullptr;
    if (h->precond) {
        if (h->nsys != 1 || nrhs != 1 || transpose || h->prec != kFP64)
            return fail(h, SFGMRES_ERR_INVALID_ARG, "ILU(0) preconditioning needs a single system, one right-hand "
                                                    "side, FP64 inner cycles and no transpose");
        if ((rc = ensure_ilu(h))) return rc;
    }
    if ((rc = get_geometry(h, nrhs, &g))) return rc;
    if ((rc = build_sketch(h, s))) return rc;
    if (transpose && (rc = ensure_transpose(h))) return rc;
    if (h->prec != kFP64 && (rc = ensure_f32(h, transpose))) return rc;
    {
        const int v = transpose ? (h->vec_opt ? h->vec_opt : h->vecT) : h->vec;
        if (v == 0 && (rc = ensure_bins(h, transpose))) return rc;
        if (v == 0 && (rc = ensure_bcopy(h, transpose))) return rc;
        if (v == 1 && h->prec == kFP64 && (rc = ensure_sell(h, transpose))) return rc;
    }
    const size_t vt = (h->prec == kFP64) ? 8 : (h->prec == kFP32 ? 4 : 2);
    const size_t at = (h->prec == kFP64) ? 8 : 4;
    const size_t N = (size_t)g->N;
    const size_t nb = (size_t)g->nblk;
    const size_t Pn = (size_t)g->P;
    const size_t M = (size_t)m, S = (size_t)s;
    if ((rc = ensure(h, h->U, (M + 1) * N * vt))) return rc;
    if ((rc = ensure(h, h->W, N * at))) return rc;
    if ((rc = ensure(h, h->sigma, Pn * (M + 1) * 8))) return rc;
    if ((rc = ensure(h, h->normpart, 2 * nb * at))) return rc;
    if ((rc = ensure(h, h->hpart, nb * kMaxTrunc * at))) return rc;
    if ((rc = ensure(h, h->cpart, nb * S * at))) return rc;
    if ((rc = ensure(h, h->C, Pn * M * S * 8))) return rc;
    if ((rc = ensure(h, h->Q, Pn * M * S * 8))) return rc;
    if ((rc = ensure(h, h->Qt, Pn * M * S * 8))) return rc;
    if ((rc = ensure(h, h->R, Pn * M * M * 8))) return rc;
    if ((rc = ensure(h, h->d, Pn * M * 8))) return rc;
    if ((rc = ensure(h, h->e, Pn * S * 8))) return rc;
    if ((rc = ensure(h, h->c0, Pn * S * 8))) return rc;
    if ((rc = ensure(h, h->rho, Pn * M * 8))) return rc;
    if ((rc = ensure(h, h->y, Pn * M * 8))) return rc;
    if ((rc = ensure(h, h->coef, Pn * M * 8))) return rc;
    if ((rc = ensure(h, h->hco, Pn * M * kMaxTrunc * 8))) return rc;
    if ((rc = ensure(h, h->cyc, Pn * sizeof(CycleState)))) return rc;
    if (jmax > 0) {
        const size_t J = (size_t)jmax;
        if ((rc = ensure(h, h->Vb, (J + 1) * N * 8))) return rc;
        if ((rc = ensure(h, h->Z, J * N * 8))) return rc;
        if ((rc = ensure(h, h->nu, Pn * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->Wo, N * 8))) return rc;
        if ((rc = ensure(h, h->opart, nb * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->h1, Pn * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->h2, Pn * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->H, Pn * (J + 1) * J * 8))) return rc;
        if ((rc = ensure(h, h->cs, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->sn, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->g, Pn * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->yo, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->est_hist, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->ffom_hist, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->ires_hist, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->rho_hist, Pn * J * 8))) return rc;
        if ((rc = ensure(h, h->k_hist, Pn * J * 4))) return rc;
        if ((rc = ensure(h, h->reason_hist, Pn * J * 4))) return rc;
    }
    if ((rc = ensure(h, h->npart, nb * 8))) return rc;
    if ((rc = ensure(h, h->npart2, nb * 8))) return rc;
    if ((rc = ensure(h, h->ost, Pn * sizeof(OuterState)))) return rc;
    if ((rc = ensure_host(h, h->h_ost, Pn * sizeof(OuterState)))) return rc;
    if ((rc = ensure_host(h, h->h_cyc, Pn * sizeof(CycleState)))) return rc;
    if ((rc = ensure_host(h, h->h_pflag, Pn * sizeof(int)))) return rc;
    std::memset(h->h_pflag.p, 0, Pn * sizeof(int));
    CK(cudaMemsetAsync(pflag_of(g), 0, Pn * sizeof(int), h->st));

    Plan& P = *p;
    plan_geometry(h, g, transpose, P);
    P.s = s;
    P.zeta = h->sk_zeta;
    P.kind = h->kind;
    P.seg = h->seg;
    P.ent = h->ent;
    P.sk_scale = (h->kind == 1) ? 1.0 : 1.0 / std::sqrt((double)h->sk_zeta);
    P.sk_headroom = h->sk_headroom;
    P.prec = h->prec;
    P.m = m;
    P.t = t;
    P.U = h->U.p;
    P.W = h->W.p;
    P.sigma = (double*)h->sigma.p;
    P.normpart = h->normpart.p;
    P.hpart = h->hpart.p;
    P.cpart = h->cpart.p;
    P.C = (double*)h->C.p;
    P.Q = (double*)h->Q.p;
    P.Qt = (double*)h->Qt.p;
    P.R = (double*)h->R.p;
    P.d = (double*)h->d.p;
    P.e = (double*)h->e.p;
    P.c0 = (double*)h->c0.p;
    P.rho = (double*)h->rho.p;
    P.y = (double*)h->y.p;
    P.coef = (double*)h->coef.p;
    P.hco = (double*)h->hco.p;
    P.cyc = (CycleState*)h->cyc.p;
    P.qr_cluster = qr_cluster_for(g->P, s, m, g->nblk, h->sms);
    P.jmax = jmax;
    P.Vb = (double*)h->Vb.p;
    P.Z = (double*)h->Z.p;
    P.nu = (double*)h->nu.p;
    P.Wo = (double*)h->Wo.p;
    P.opart = (double*)h->opart.p;
    P.npart = (double*)h->npart.p;
    P.npart2 = (double*)h->npart2.p;
    P.h1 = (double*)h->h1.p;
    P.h2 = (double*)h->h2.p;
    P.H = (double*)h->H.p;
    P.cs = (double*)h->cs.p;
    P.sn = (double*)h->sn.p;
    P.g = (double*)h->g.p;
    P.yo = (double*)h->yo.p;
    P.est_hist = (double*)h->est_hist.p;
    P.ffom_hist = (double*)h->ffom_hist.p;
    P.ires_hist = (double*)h->ires_hist.p;
    P.rho_hist = (double*)h->rho_hist.p;
    P.k_hist = (int*)h->k_hist.p;
    P.reason_hist = (int*)h->reason_hist.p;
    P.ost = (OuterState*)h->ost.p;
    P.sms = h->sms;
    P.gwait_extra = h->wait_extra;
    P.outer_variant = h->outer_variant;
    if (h->fuse_step) {
        if ((rc = ensure(h, h->gsync, 4 * sizeof(unsigned long long)))) return rc;
        P.gsync = (unsigned long long*)h->gsync.p;
    } else {
        P.gsync = nullptr;
    }
    if (h->precond) {
        P.ilu = h->ilu.dev;
        P.ilu_host = &h->ilu;
        P.xin = (const double*)h->ilu_t.p;
    }
    if (geo_out) *geo_out = g;
    return 0;
}

int check_params(sfgmres_ctx* h, int m, int s, int t) {
    if (m < 1 || m > kMaxM) return fail(h, SFGMRES_ERR_INVALID_ARG, "m must be in [1, 1024]");
    if (t < 0 || t > kMaxTrunc) return fail(h, SFGMRES_ERR_INVALID_ARG, "k (truncation) must be in [0, 8]");
    if (h->kind == 1) {
        if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "identity sketch needs a single-system handle");
        if (s != h->n) return fail(h, SFGMRES_ERR_INVALID_ARG, "identity sketch needs s == n");
        if (s > kMaxS) return fail(h, SFGMRES_ERR_INVALID_ARG, "identity sketch needs n <= 4096");
    } else {
        if (s < h->zeta || s > kMaxS) return fail(h, SFGMRES_ERR_INVALID_ARG, "s must be in [zeta, 4096]");
    }
    if (m > s) return fail(h, SFGMRES_ERR_INVALID_ARG, "m must not exceed s");
    return 0;
}

// ---- profiling helpers ----
// Pairs [base, base + count) of all three pools exist afterwards.
int ev_reserve(sfgmres_ctx* h, size_t base, size_t count) {
    for (auto* pool : {&h->ev_spmv, &h->ev_axpy, &h->ev_qr})
        while (pool->size() < base + count) {
            EventPair e;
            CK(cudaEventCreate(&e.a));
            if (cudaEventCreate(&e.b) != cudaSuccess) {
                cudaEventDestroy(e.a);
                CK(cudaGetLastError());
            }
            pool->push_back(e);
        }
    return 0;
}
// Records one event; inside a stream capture it becomes an event-record node of the graph, so the graph's replays
// time the kernels too.
void ev_rec(cudaEvent_t e, cudaStream_t st, bool capturing) {
    if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}
double ev_sum(const std::vector<EventPair>& pool, size_t base, size_t count) {
    double tot = 0.0;
    for (size_t i = base; i < base + count; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pool[i].a, pool[i].b) == cudaSuccess) tot += ms;
    }
    return tot;
}

// One inner cycle (Section 3) for every active problem on u_0 = vscale_p * v; j >= 0 inside a solve (C3 as
// configured), j < 0 standalone.  The sketched-QR update of step i runs on the side stream after step i's sketch
// column is ready, overlapping the next step's SpMV; the main stream waits for the last QR update before the
// least-squares solve.
// ev: base event pair of this cycle's launches (profiling), or SIZE_MAX; capturing: inside a stream capture.
int run_cycle(sfgmres_ctx* h, const Plan& P, int j, const double* v, const double* vscale, int vstride, int c3,
              double* z, size_t ev = SIZE_MAX, bool capturing = false) {
    launch_cycle_start(P, j, v, vscale, vstride, c3, h->cond_thr);
    // profile 1: events around every inner-kernel launch; profile 2: one pair of events around the cycle's chain of
    // step launches on the step stream (pair ev: before step 0, after step m - 1), nothing between the launches
    const bool prof = (ev != SIZE_MAX) && h->profile == 1;
    const bool span = (ev != SIZE_MAX) && h->profile == 2;
    h->step_fused = false;
    for (int i = 0; i < P.m; ++i) {
        const bool last = (i == P.m - 1);
        // right preconditioning: the step multiplies t_i = M^{-1} u_i (the passes return at once after a stop)
        if (P.ilu_host) launch_ilu_apply(P, i, (const double*)P.U + (int64_t)i * P.N, const_cast<double*>(P.xin));
        if (prof || (span && i == 0)) ev_rec(h->ev_spmv[ev + i].a, h->st, capturing);
        const bool fused = launch_inner_step(P, i, last);  // one launch, timed as the inner kernel
        if (!fused) launch_inner_spmv(P, i);
        if (prof) ev_rec(h->ev_spmv[ev + i].b, h->st, capturing);
        if (!fused) {
            if (prof) ev_rec(h->ev_axpy[ev + i].a, h->st, capturing);
            launch_inner_axpy(P, i, last);
            if (prof) ev_rec(h->ev_axpy[ev + i].b, h->st, capturing);
        }
        if (span && last) ev_rec(h->ev_spmv[ev].b, h->st, capturing);
        h->step_fused |= fused;
        CK(cudaEventRecord(h->ev_c, h->st));
        CK(cudaStreamWaitEvent(h->qst, h->ev_c, 0));
        if (prof) ev_rec(h->ev_qr[ev + i].a, h->qst, capturing);
        CK(launch_inner_qr(P, i, h->qst));
        if (prof) ev_rec(h->ev_qr[ev + i].b, h->qst, capturing);
    }
    CK(cudaEventRecord(h->ev_q, h->qst));
    CK(cudaStreamWaitEvent(h->st, h->ev_q, 0));
    if (P.ilu_host) {  // z = M^{-1} (B_k y)
        launch_inner_finish(P, (double*)h->ilu_zt.p);
        launch_ilu_apply(P, -1, (const double*)h->ilu_zt.p, z);
    } else {
        launch_inner_finish(P, z);
    }
    return 0;
}

// Everything a captured outer step depends on: the plan's pointers and sizes and the cycle options.
std::vector<uint64_t> plan_key(const sfgmres_ctx* h, const Plan& P) {
    std::vector<uint64_t> k;
    auto u = [&](const void* p) { k.push_back((uint64_t)(uintptr_t)p); };
    for (const void* p : std::initializer_list<const void*>{(const void*)P.perm, (const void*)P.cls,
                                                            (const void*)P.rp, (const void*)P.col, (const void*)P.val, (const void*)P.val32,
                          (const void*)P.blk_v0, (const void*)P.seg, (const void*)P.sl_off, (const void*)P.sl_col,
                          (const void*)P.sl_val, (const void*)P.sl_base, (const void*)P.sl_len, (const void*)P.ent, P.U, P.W,
                          (const void*)P.sigma, P.normpart, P.hpart, P.cpart, (const void*)P.C, (const void*)P.Q, (const void*)P.Qt,
                          (const void*)P.R, (const void*)P.d, (const void*)P.e, (const void*)P.c0,
                          (const void*)P.rho, (const void*)P.y, (const void*)P.coef, (const void*)P.hco,
                          (const void*)P.cyc, (const void*)P.Vb, (const void*)P.Z, (const void*)P.nu,
                          (const void*)P.Wo, (const void*)P.opart, (const void*)P.npart, (const void*)P.npart2,
                          (const void*)P.h1, (const void*)P.h2, (const void*)P.H, (const void*)P.cs,
                          (const void*)P.sn, (const void*)P.g, (const void*)P.yo, (const void*)P.est_hist,
                          (const void*)P.ffom_hist, (const void*)P.ires_hist, (const void*)P.rho_hist,
                          (const void*)P.k_hist, (const void*)P.reason_hist,
                          (const void*)P.ost, (const void*)P.st, (const void*)h->qst, (const void*)P.gsync,
                          (const void*)P.xin, (const void*)P.ilu.lu, (const void*)P.brp, (const void*)P.bcol,
                          (const void*)P.bval})
        u(p);
    for (int64_t v : std::initializer_list<int64_t>{(int64_t)P.nnz, (int64_t)P.vec, (int64_t)P.N, (int64_t)P.P, (int64_t)P.nblk, (int64_t)P.Bn,
                      (int64_t)P.s, (int64_t)P.zeta, (int64_t)P.kind, (int64_t)P.sk_headroom, (int64_t)P.prec,
                      (int64_t)P.m, (int64_t)P.t, (int64_t)P.qr_cluster, (int64_t)P.jmax, (int64_t)h->c3,
                      (int64_t)h->profile, (int64_t)P.gwait_extra, (int64_t)P.outer_variant})
        k.push_back((uint64_t)v);
    uint64_t bits;
    std::memcpy(&bits, &P.sk_scale, 8);
    k.push_back(bits);
    std::memcpy(&bits, &h->cond_thr, 8);
    k.push_back(bits);
    return k;
}

void drop_graphs(sfgmres_ctx* h) {
    for (cudaGraphExec_t g : h->graph_exec)
        if (g) cudaGraphExecDestroy(g);
    h->graph_exec.clear();
    h->graph_launches.clear();
    h->graph_key.clear();
    h->graph_ev.clear();
    h->ev_graph = 0;
}

// One outer step j (inner cycle j and the outer FGMRES update) for every active problem.  With graphs on, the step
// is captured from the handle's streams once per plan and j, then replayed as a single graph launch.  With profiling
// on, the step's inner-kernel launches are bracketed by events (event-record nodes of the graph).
int outer_step(sfgmres_ctx* h, const Plan& P, int j) {
    auto enqueue = [&](size_t ev, bool capturing) -> int {
        int rc = run_cycle(h, P, j, P.Vb + (int64_t)j * P.N, P.nu + j, P.jmax + 1, h->c3, P.Z + (int64_t)j * P.N,
                           ev, capturing);
        if (rc) return rc;
        launch_outer_step(P, j);
        return 0;
    };
    const bool prof = h->profile != 0;
    auto take_events = [&](size_t& ev) -> int {
        ev = SIZE_MAX;
        if (!prof) return 0;
        int rc = ev_reserve(h, h->ev_next, (size_t)P.m);
        if (rc) return rc;
        ev = h->ev_next;
        h->ev_next += (size_t)P.m;
        h->ev_steps.push_back({j, ev});
        return 0;
    };
    int rc;
    if (!h->use_graph) {
        size_t ev;
        if ((rc = take_events(ev))) return rc;
        return enqueue(ev, false);
    }
    std::vector<uint64_t> key = plan_key(h, P);
    if (key != h->graph_key) {
        drop_graphs(h);
        h->graph_key = key;
        h->ev_next = 0;
    }
    if ((int)h->graph_exec.size() <= j) {
        h->graph_exec.resize(j + 1, nullptr);
        h->graph_launches.resize(j + 1, 0);
        h->graph_ev.resize(j + 1, SIZE_MAX);
    }
    if (!h->graph_exec[j]) {
        const int64_t l0 = g_launches;
        // a graph's events stay its own: pairs after every cached graph's, below those of one-by-one launches
        h->ev_next = h->ev_graph;
        size_t ev;
        if ((rc = take_events(ev))) return rc;
        if (prof) h->ev_steps.pop_back();  // recorded below, once the graph exists
        CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
        rc = enqueue(ev, true);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CK(e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        h->graph_exec[j] = ex;
        h->graph_launches[j] = g_launches - l0;
        h->graph_ev[j] = ev;
        if (prof) h->ev_graph = h->ev_next;
        g_launches = l0;
    }
    if (h->graph_ev[j] != SIZE_MAX) h->ev_steps.push_back({j, h->graph_ev[j]});
    CK(cudaGraphLaunch(h->graph_exec[j], h->st));
    g_launches += h->graph_launches[j];
    return 0;
}

// Per-problem outcome of a solve.
struct ProbOut {
    int status = SFGMRES_NOT_CONVERGED;
    int outer = 0;
    double rel_true = 0.0, rel_est = 0.0;
    bool done = false, brk = false, nan_init = false, sync_fail = false;
};

struct SolveOut {
    std::vector<ProbOut> pr;
    int jmax = 0;
    Plan P;
};

int status_of(const std::vector<ProbOut>& pr) {
    bool nc = false, brk = false, nan = false, cuda = false;
    for (const ProbOut& o : pr) {
        cuda |= (o.status == SFGMRES_ERR_CUDA);
        nan |= (o.status == SFGMRES_ERR_NAN);
        nc |= (o.status == SFGMRES_NOT_CONVERGED);
        brk |= (o.status == SFGMRES_BREAKDOWN);
    }
    if (cuda) return SFGMRES_ERR_CUDA;
    if (nan) return SFGMRES_ERR_NAN;
    if (nc) return SFGMRES_NOT_CONVERGED;
    if (brk) return SFGMRES_BREAKDOWN;
    return SFGMRES_OK;
}

// The solve of every problem of the batch: b, x0, x hold nrhs * n values in problem order.
int solve_core(sfgmres_t h, bool transpose, int nrhs, const double* b, const double* x0, double* x, int m, int s,
               int k, double tol, SolveOut* so) {
    const int jmax = h->max_outer;
    Plan P;
    Geo* g = nullptr;
    int rc;
    if ((rc = prepare(h, nrhs, m, s, k, jmax, &P, &g, transpose))) return rc;
    const int NP = P.P;
    const size_t nbytes = (size_t)P.N * sizeof(double);
    if ((rc = ensure(h, h->bst, nbytes))) return rc;
    if ((rc = ensure(h, h->xst, nbytes))) return rc;
    if ((rc = ensure(h, h->x0st, nbytes))) return rc;
    double* db = (double*)h->bst.p;
    double* dx = (double*)h->xst.p;
    double* dx0 = (double*)h->x0st.p;
    int* hflag = (int*)h->h_pflag.p;
    int* dflag = pflag_of(g);
    OuterState* host_ost = (OuterState*)h->h_ost.p;
    const bool x_dev = is_device_ptr(x);
    h->ev_steps.clear();
    h->ev_next = h->ev_graph;  // one-by-one launches reuse the pairs after the cached graphs'
    CK(cudaEventRecord(h->ev_t0, h->st));
    // private copies of b and x0 (x may alias x0, and host inputs are staged)
    CK(cudaMemcpyAsync(db, b, nbytes, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (x0) {
        CK(cudaMemcpyAsync(dx0, x0, nbytes, is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           h->st));
    }
    const double* px0 = x0 ? dx0 : nullptr;
    // every problem's iterate starts at x0; finalisation overwrites the problems it covers
    if (x0) k_copy<<<grid_for(P.N), 256, 0, h->st>>>(P.N, dx0, dx);
    else k_fill<<<grid_for(P.N), 256, 0, h->st>>>(P.N, 0.0, dx);
    ++g_launches;
    // r0 = b - A x0 into v_0; beta, ||b||
    launch_residual(P, db, px0, P.Vb, false);
    launch_init_state(P, tol);
    CK(cudaMemcpyAsync(host_ost, P.ost, NP * sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    so->pr.assign(NP, ProbOut());
    so->jmax = jmax;
    std::vector<ProbOut>& pr = so->pr;
    int active = 0;
    bool any_zero = false;
    for (int p = 0; p < NP; ++p) {
        const OuterState& os = host_ost[p];
        ProbOut& o = pr[p];
        if (!std::isfinite(os.beta) || !std::isfinite(os.bnorm) || os.nan) {
            o.status = SFGMRES_ERR_NAN;
            o.nan_init = true;
            o.done = true;
        } else if (os.bnorm == 0.0) {  // x = 0
            o.status = SFGMRES_OK;
            o.done = true;
            hflag[p] |= 4;
            any_zero = true;
        } else if (os.beta <= os.tol_abs) {  // x0 already meets the tolerance
            o.status = SFGMRES_OK;
            o.done = true;
            o.rel_true = o.rel_est = os.beta / os.bnorm;
        } else {
            ++active;
        }
        if (o.done) hflag[p] |= 1;
    }
    if (active < NP) {
        CK(cudaMemcpyAsync(dflag, hflag, NP * sizeof(int), cudaMemcpyHostToDevice, h->st));
        if (any_zero) {
            k_zero_flagged<<<P.nblk, 256, 0, h->st>>>(P, dx);
            ++g_launches;
        }
    }
    std::vector<int> fin;
    for (int j = 0; j < jmax && active > 0; ++j) {
        if ((rc = outer_step(h, P, j))) return rc;
        CK(cudaMemcpyAsync(host_ost, P.ost, NP * sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        CK(cudaGetLastError());
        const bool last = (j + 1 == jmax);
        fin.clear();
        bool changed = false;
        for (int p = 0; p < NP; ++p) {
            ProbOut& o = pr[p];
            if (o.done) continue;
            const OuterState& os = host_ost[p];
            if (os.nan) {
                o.status = os.sync_fail ? SFGMRES_ERR_CUDA : SFGMRES_ERR_NAN;
                o.sync_fail = os.sync_fail != 0;
                o.done = true;
                hflag[p] |= 1;
                changed = true;
                --active;
                continue;
            }
            if (os.breakdown == 2) {  // the inner cycle accepted no column: keep the iterate of step j
                o.brk = true;
                o.outer = j;
                fin.push_back(p);
                continue;
            }
            o.outer = j + 1;
            o.rel_est = os.est / os.bnorm;
            if (os.conv_est || os.breakdown == 1 || last) fin.push_back(p);
        }
        if (!fin.empty()) {
            for (int p : fin) hflag[p] |= 2;
            CK(cudaMemcpyAsync(dflag, hflag, NP * sizeof(int), cudaMemcpyHostToDevice, h->st));
            launch_final_x(P, jmax, px0, dx);
            launch_residual(P, db, dx, nullptr, true);
            launch_true_residual_reduce(P);
            CK(cudaMemcpyAsync(host_ost, P.ost, NP * sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            CK(cudaGetLastError());
            for (int p : fin) {
                ProbOut& o = pr[p];
                const OuterState& os = host_ost[p];
                o.rel_true = std::sqrt(os.true_res2) / os.bnorm;
                hflag[p] &= ~2;
                if (o.brk) o.status = SFGMRES_BREAKDOWN;
                else if (o.rel_true <= tol || os.breakdown == 1) o.status = SFGMRES_OK;
                else if (last) o.status = SFGMRES_NOT_CONVERGED;
                else continue;
                o.done = true;
                hflag[p] |= 1;
                --active;
            }
            changed = true;
        }
        if (changed) CK(cudaMemcpyAsync(dflag, hflag, NP * sizeof(int), cudaMemcpyHostToDevice, h->st));
    }
    CK(cudaMemcpyAsync(x, dx, nbytes, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaEventRecord(h->ev_t1, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    so->P = P;
    return 0;
}

int check_solve_args(sfgmres_t h, const double* b, double* x, int m, int s, int k, double tol) {
    if (!b || !x) return fail(h, SFGMRES_ERR_INVALID_ARG, "b and x must not be NULL");
    if (!(tol > 0.0 && tol < 1.0)) return fail(h, SFGMRES_ERR_INVALID_ARG, "tol must be in (0, 1)");
    return check_params(h, m, s, k);
}

int solve_single(sfgmres_t h, bool transpose, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                 int32_t k, double tol, sfgmres_stats* st) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "this handle holds several systems: use sfgmres_solve_batch");
    int rc = check_solve_args(h, b, x, m, s, k, tol);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int64_t launches0 = g_launches;
    SolveOut so;
    if ((rc = solve_core(h, transpose, 1, b, x0, x, m, s, k, tol, &so))) return rc;
    const ProbOut& o = so.pr[0];
    const int status = o.status;
    if (status == SFGMRES_ERR_CUDA) return fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
    if (status == SFGMRES_ERR_NAN) {
        return fail(h, SFGMRES_ERR_NAN, o.nan_init ? "non-finite value in b or x0 (or in A x0)"
                                                   : "non-finite value during the iteration");
    }
    if (st) {
        const Plan& P = so.P;
        const int jmax = so.jmax;
        st->status = status;
        st->outer_iters = o.outer;
        st->rel_res_true = o.rel_true;
        st->rel_res_est = o.rel_est;
        const int cnt = std::min(o.outer + (status == SFGMRES_BREAKDOWN ? 1 : 0), jmax);
        std::vector<int> kh(std::max(cnt, 1)), rh(std::max(cnt, 1));
        std::vector<double> eh(std::max(cnt, 1)), fh(std::max(cnt, 1)), ih(std::max(cnt, 1)), qh(std::max(cnt, 1));
        if (cnt > 0) {
            CK(cudaMemcpy(kh.data(), P.k_hist, cnt * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(rh.data(), P.reason_hist, cnt * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(eh.data(), P.est_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fh.data(), P.ffom_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(ih.data(), P.ires_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(qh.data(), P.rho_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
        }
        int tot = 0;
        for (int q = 0; q < cnt; ++q) tot += kh[q];
        st->total_inner = tot;
        const int cap = std::min(cnt, st->hist_cap);
        for (int q = 0; q < cap; ++q) {
            if (st->inner_k) st->inner_k[q] = kh[q];
            if (st->inner_reason) st->inner_reason[q] = rh[q];
            if (st->res_est && q < o.outer) st->res_est[q] = eh[q];
            if (st->ffom_res && q < o.outer) st->ffom_res[q] = fh[q];
            if (st->inner_res && q < o.outer) st->inner_res[q] = ih[q];
            if (st->inner_rho && q < o.outer) st->inner_rho[q] = qh[q];
        }
        st->kernel_launches = g_launches - launches0;
        float tms = 0.f;
        cudaEventElapsedTime(&tms, h->ev_t0, h->ev_t1);
        st->t_total_ms = tms;
        st->t_step_span_ms = 0.0;
        st->n_step_span = 0;
        if (h->profile == 2) {
            // the cycles whose m step launches all built a basis vector, timed from before the first launch to after
            // the last (fused single launches on the step stream only)
            st->t_inner_spmv_ms = st->t_inner_axpy_ms = st->t_qr_ms = 0.0;
            st->n_inner_spmv = st->n_inner_axpy = st->n_qr = 0;
            if (h->step_fused && !P.ilu_host)
                for (const auto& js : h->ev_steps) {
                    if (js.first >= cnt || kh[js.first] != P.m) continue;
                    st->t_step_span_ms += ev_sum(h->ev_spmv, js.second, 1);
                    st->n_step_span += P.m;
                }
        } else if (h->profile) {
            // the launches of inner steps i < k_j of each outer step j (those that built a basis vector); the
            // launches after the cycle stopped only read the stop flag and return
            st->t_inner_spmv_ms = st->t_inner_axpy_ms = st->t_qr_ms = 0.0;
            st->n_inner_spmv = st->n_inner_axpy = st->n_qr = 0;
            for (const auto& js : h->ev_steps) {
                if (js.first >= cnt) continue;
                const size_t kw = (size_t)std::max(0, std::min(kh[js.first], P.m));
                st->t_inner_spmv_ms += ev_sum(h->ev_spmv, js.second, kw);
                st->t_qr_ms += ev_sum(h->ev_qr, js.second, kw);
                st->n_inner_spmv += (int64_t)kw;
                if (!h->step_fused) {
                    st->t_inner_axpy_ms += ev_sum(h->ev_axpy, js.second, kw);
                    st->n_inner_axpy += (int64_t)kw;
                }
                st->n_qr += (int64_t)kw;
            }
        } else {
            st->t_inner_spmv_ms = st->t_inner_axpy_ms = st->t_qr_ms = 0.0;
            st->n_inner_spmv = st->n_inner_axpy = st->n_qr = 0;
        }
    }
    return status;
}

}  // namespace

// =====================================================================================================================
extern "C" {

const char* sfgmres_version(void) { return "sfgmres-gb300 0.2 (sm_103a)"; }

const char* sfgmres_last_error(sfgmres_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int sfgmres_create_batch(sfgmres_t* out, int32_t nsys, const int64_t* sys_n, int64_t nnz, const int64_t* row_ptr,
                         const int32_t* col_idx, const double* vals, uint64_t sketch_seed, int32_t flags,
                         void* stream) {
    sfgmres_ctx* h = nullptr;
    if (!out) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || !sys_n) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "nsys must be >= 1 and sys_n not NULL");
    int64_t n = 0;
    for (int q = 0; q < nsys; ++q) {
        if (sys_n[q] < 1) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "every system needs at least one row");
        n += sys_n[q];
        if (n > INT32_MAX - 1) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "total rows must be below 2^31 - 1");
    }
    if (nnz < 0 || nnz > INT32_MAX) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "nnz must be in [0, 2^31-1]");
    if (!row_ptr || (nnz > 0 && (!col_idx || !vals)))
        return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "NULL CSR array");
    h = new sfgmres_ctx();
    h->nsys = nsys;
    h->n = (int)n;
    h->nnz = nnz;
    h->seed = sketch_seed;
    h->sys_n.resize(nsys);
    h->sys_moff.resize(nsys + 1);
    {
        int off = 0;
        for (int q = 0; q < nsys; ++q) {
            h->sys_n[q] = (int)sys_n[q];
            h->sys_moff[q] = off;
            off += (int)sys_n[q];
        }
        h->sys_moff[nsys] = off;
    }
    cudaError_t ce = cudaGetDevice(&h->dev);
    if (ce != cudaSuccess) {
        delete h;
        return fail(nullptr, SFGMRES_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
    if (stream) {
        h->st = (cudaStream_t)stream;
    } else {
        cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    auto bail = [&](int code, const std::string& msg) {
        g_create_error = msg;
        sfgmres_destroy(h);
        return code;
    };
    const bool host = (flags & SFGMRES_CSR_HOST) != 0;
    int64_t* rp64 = nullptr;
    int* bad = nullptr;
    int* dmoff = nullptr;
    if (cudaMalloc(&h->rp, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->col, std::max<int64_t>(nnz, 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->val, std::max<int64_t>(nnz, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&rp64, (n + 1) * sizeof(int64_t)) != cudaSuccess || cudaMalloc(&bad, 2 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&dmoff, (nsys + 1) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (rp64) cudaFree(rp64);
        if (bad) cudaFree(bad);
        if (dmoff) cudaFree(dmoff);
        return bail(SFGMRES_ERR_OOM, "out of device memory for the CSR copy");
    }
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaMemcpyAsync(rp64, row_ptr, (n + 1) * sizeof(int64_t), kind, h->st);
    if (nnz > 0) {
        cudaMemcpyAsync(h->col, col_idx, nnz * sizeof(int), kind, h->st);
        cudaMemcpyAsync(h->val, vals, nnz * sizeof(double), kind, h->st);
    }
    cudaMemcpyAsync(dmoff, h->sys_moff.data(), (nsys + 1) * sizeof(int), cudaMemcpyHostToDevice, h->st);
    cudaMemsetAsync(bad, 0, 2 * sizeof(int), h->st);
    const int64_t cover = std::max<int64_t>(n + 1, nnz);
    k_validate_csr<<<(int)((cover + 255) / 256), 256, 0, h->st>>>((int)n, nnz, rp64, h->col, h->rp, bad, dmoff,
                                                                  nsys);
    int hbad2[2] = {0, 0};
    cudaMemcpyAsync(hbad2, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st);
    ce = cudaStreamSynchronize(h->st);
    cudaFree(rp64);
    cudaFree(bad);
    cudaFree(dmoff);
    if (ce != cudaSuccess) return bail(SFGMRES_ERR_CUDA, std::string("CSR upload: ") + cudaGetErrorString(ce));
    const int hbad = hbad2[0];
    h->maxlen = hbad2[1];
    if (hbad) {
        char buf[200];
        snprintf(buf, sizeof buf, "invalid CSR (code %d: 1 range, 2 row_ptr[0]!=0, 4 row_ptr[n]!=nnz, "
                 "8 decreasing row_ptr, 16 column out of range, 32 column outside the row's system)", hbad);
        return bail(SFGMRES_ERR_INVALID_ARG, buf);
    }
    set_list_geometry(h);
    h->vec = choose_vec(nnz, h->n, h->maxlen);
    cudaEventCreate(&h->ev_t0);
    cudaEventCreate(&h->ev_t1);
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (cudaStreamCreateWithPriority(&h->qst, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_c, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_q, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(SFGMRES_ERR_CUDA, "stream/event creation failed");
    }
    *out = h;
    return SFGMRES_OK;
}

int sfgmres_create(sfgmres_t* out, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* vals, uint64_t sketch_seed, int32_t flags, void* stream) {
    if (out) *out = nullptr;
    if (n < 1 || n > INT32_MAX - 1) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "n must be in [1, 2^31-2]");
    return sfgmres_create_batch(out, 1, &n, nnz, row_ptr, col_idx, vals, sketch_seed, flags, stream);
}

int sfgmres_destroy(sfgmres_t h) {
    if (!h) return SFGMRES_OK;
    if (h->st) cudaStreamSynchronize(h->st);
    cudaFree(h->rp);
    cudaFree(h->col);
    cudaFree(h->val);
    if (h->val32) cudaFree(h->val32);
    for (void* q : {(void*)h->rpT, (void*)h->colT, (void*)h->srcT, (void*)h->valT, (void*)h->val32T})
        if (q) cudaFree(q);
    if (h->seg) cudaFree(h->seg);
    if (h->ent) cudaFree(h->ent);
    for (int t = 0; t < 2; ++t) {
        if (h->perm[t]) cudaFree(h->perm[t]);
        if (h->cls[t]) cudaFree(h->cls[t]);
    }
    if (h->lb) cudaFree(h->lb);
    for (auto& B : h->bc)
        for (void* q : {(void*)B.rp, (void*)B.col, (void*)B.val})
            if (q) cudaFree(q);
    for (auto& S : h->sell)
        for (void* q : {(void*)S.off, (void*)S.len, (void*)S.col, (void*)S.val})
            if (q) cudaFree(q);
    if (h->sl_sys) cudaFree(h->sl_sys);
    if (h->sl_base) cudaFree(h->sl_base);
    DevBuf* bufs[] = {&h->U, &h->W, &h->sigma, &h->normpart, &h->hpart, &h->cpart, &h->C, &h->Q, &h->Qt, &h->R, &h->d,
                      &h->e, &h->c0, &h->rho, &h->y, &h->coef, &h->hco, &h->cyc, &h->Vb, &h->Z, &h->nu, &h->Wo,
                      &h->opart, &h->npart, &h->npart2, &h->h1, &h->h2, &h->H, &h->cs, &h->sn, &h->g, &h->yo,
                      &h->est_hist, &h->ffom_hist, &h->ires_hist, &h->rho_hist, &h->k_hist, &h->reason_hist, &h->ost, &h->bst, &h->xst,
                      &h->x0st, &h->gsync};
    for (DevBuf* b : bufs) release(*b);
    for (DevBuf* b : {&h->ilu_rp, &h->ilu_col, &h->ilu_diag, &h->ilu_perm, &h->ilu_src_d, &h->ilu_lu, &h->ilu_y,
                      &h->ilu_zp, &h->ilu_t, &h->ilu_zt, &h->ilu_bad})
        release(*b);
    for (auto& L : h->lvl)
        for (DevBuf* b : {&L.Vb, &L.Z, &L.nu, &L.Wo, &L.opart, &L.npart, &L.npart2, &L.h1, &L.h2, &L.H, &L.cs, &L.sn,
                          &L.g, &L.yo, &L.est_hist, &L.ffom_hist, &L.ires_hist, &L.rho_hist, &L.k_hist,
                          &L.reason_hist, &L.ost, &L.pflag, &L.rhs})
            release(*b);
    for (Geo& g : h->geos) {
        release(g.tab);
    }
    drop_graphs(h);
    release_host(h->h_ost);
    release_host(h->h_cyc);
    release_host(h->h_pflag);
    for (auto* pool : {&h->ev_spmv, &h->ev_axpy, &h->ev_qr})
        for (auto& e : *pool) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    if (h->ev_c) cudaEventDestroy(h->ev_c);
    if (h->ev_q) cudaEventDestroy(h->ev_q);
    if (h->qst) {
        cudaStreamSynchronize(h->qst);
        cudaStreamDestroy(h->qst);
    }
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
    return SFGMRES_OK;
}

int sfgmres_set_option(sfgmres_t h, int32_t key, double v) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    const int iv = (int)v;
    switch (key) {
        case SFGMRES_OPT_PRECISION:
            if (iv < 0 || iv > 2 || iv != v) return fail(h, SFGMRES_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
            if (iv != h->prec) {
                h->prec = iv;
                if (h->nsys == 1 && !h->block_rows) set_list_geometry(h);  // the default row blocks depend on it
            }
            return 0;
        case SFGMRES_OPT_ZETA:
            if (iv < 1 || iv > kMaxZeta || iv != v) return fail(h, SFGMRES_ERR_INVALID_ARG, "zeta must be 1..16");
            h->zeta = iv;
            return 0;
        case SFGMRES_OPT_COND_THRESHOLD:
            if (!(v > 1.0)) return fail(h, SFGMRES_ERR_INVALID_ARG, "cond threshold must exceed 1");
            h->cond_thr = v;
            return 0;
        case SFGMRES_OPT_C3:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "C3 must be 0 or 1");
            h->c3 = iv;
            return 0;
        case SFGMRES_OPT_MAX_OUTER:
            if (iv < 1 || iv > 1000 || iv != v) return fail(h, SFGMRES_ERR_INVALID_ARG, "max_outer must be 1..1000");
            h->max_outer = iv;
            return 0;
        case SFGMRES_OPT_SKETCH_KIND:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sketch kind must be 0 or 1");
            h->kind = iv;
            return 0;
        case SFGMRES_OPT_PROFILE:
            if (iv < 0 || iv > 2) return fail(h, SFGMRES_ERR_INVALID_ARG, "profile must be 0, 1 or 2");
            h->profile = iv;
            return 0;
        case SFGMRES_OPT_SPMV_VECTOR:
            if (!(iv == 0 || iv == 2 || iv == 4 || iv == 8 || iv == 16 || iv == 32) || iv != v)
                return fail(h, SFGMRES_ERR_INVALID_ARG, "spmv vector width must be 0, 2, 4, 8, 16 or 32");
            h->vec_opt = iv;
            h->vec = iv ? iv : choose_vec(h->nnz, h->n, h->maxlen);
            return 0;
        case SFGMRES_OPT_FUSED_STEP:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "fused step must be 0 or 1");
            h->fuse_step = iv;
            return 0;
        case SFGMRES_OPT_STEP_WAIT_EXTRA:
            if (iv != v || iv < 0 || iv > 1024) return fail(h, SFGMRES_ERR_INVALID_ARG, "step wait extra must be 0..1024");
            h->wait_extra = iv;
            return 0;
        case SFGMRES_OPT_OUTER_VARIANT:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "outer variant must be 0 or 1");
            h->outer_variant = iv;
            return 0;
        case SFGMRES_OPT_PRECOND:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "precond must be 0 or 1");
            h->precond = iv;
            return 0;
        case SFGMRES_OPT_GRAPH:
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "graph must be 0 or 1");
            h->use_graph = iv;
            return 0;
        case SFGMRES_OPT_BLOCK_ROWS:
            if (iv != v || !(iv == 0 || (iv >= 32 && iv <= kBlockRowsMax && iv % 32 == 0)))
                return fail(h, SFGMRES_ERR_INVALID_ARG, "block rows must be 0 or a multiple of 32 in [32, 8192]");
            if (iv != h->block_rows) {
                h->block_rows = iv;
                set_list_geometry(h);
            }
            return 0;
        default:
            return fail(h, SFGMRES_ERR_INVALID_ARG, "unknown option key");
    }
}

int sfgmres_get_option(sfgmres_t h, int32_t key, double* v) {
    if (!h || !v) return SFGMRES_ERR_INVALID_ARG;
    switch (key) {
        case SFGMRES_OPT_PRECISION: *v = h->prec; return 0;
        case SFGMRES_OPT_ZETA: *v = h->zeta; return 0;
        case SFGMRES_OPT_COND_THRESHOLD: *v = h->cond_thr; return 0;
        case SFGMRES_OPT_C3: *v = h->c3; return 0;
        case SFGMRES_OPT_MAX_OUTER: *v = h->max_outer; return 0;
        case SFGMRES_OPT_SKETCH_KIND: *v = h->kind; return 0;
        case SFGMRES_OPT_PROFILE: *v = h->profile; return 0;
        case SFGMRES_OPT_SPMV_VECTOR: *v = h->vec; return 0;
        case SFGMRES_OPT_BLOCK_ROWS: *v = h->sys_Bq.empty() ? 0 : h->sys_Bq[0]; return 0;
        case SFGMRES_OPT_GRAPH: *v = h->use_graph; return 0;
        case SFGMRES_OPT_FUSED_STEP: *v = h->fuse_step; return 0;
        case SFGMRES_OPT_STEP_WAIT_EXTRA: *v = h->wait_extra; return 0;
        case SFGMRES_OPT_OUTER_VARIANT: *v = h->outer_variant; return 0;
        case SFGMRES_OPT_PRECOND: *v = h->precond; return 0;
        default: return fail(h, SFGMRES_ERR_INVALID_ARG, "unknown option key");
    }
}

int sfgmres_solve(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s, int32_t k,
                  double tol, sfgmres_stats* st) {
    return solve_single(h, false, b, x0, x, m, s, k, tol, st);
}

int sfgmres_solve_transpose(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                            int32_t k, double tol, sfgmres_stats* st) {
    return solve_single(h, true, b, x0, x, m, s, k, tol, st);
}

int sfgmres_solve_batch(sfgmres_t h, int32_t nrhs, const double* b, const double* x0, double* x, int32_t m,
                        int32_t s, int32_t k, double tol, int32_t flags, sfgmres_batch_stats* st) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (nrhs < 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "nrhs must be >= 1");
    if (flags & ~SFGMRES_SOLVE_TRANSPOSE) return fail(h, SFGMRES_ERR_INVALID_ARG, "unknown solve flag");
    int rc = check_solve_args(h, b, x, m, s, k, tol);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int64_t launches0 = g_launches;
    SolveOut so;
    if ((rc = solve_core(h, (flags & SFGMRES_SOLVE_TRANSPOSE) != 0, nrhs, b, x0, x, m, s, k, tol, &so))) return rc;
    const int status = status_of(so.pr);
    if (status == SFGMRES_ERR_CUDA) fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
    if (status == SFGMRES_ERR_NAN) {
        int first = 0;
        while (so.pr[first].status != SFGMRES_ERR_NAN) ++first;
        fail(h, SFGMRES_ERR_NAN, "non-finite value in problem " + std::to_string(first) +
                                     " (its x is x0; the other problems' results are valid)");
    }
    if (st) {
        const int NP = (int)so.pr.size();
        st->problems = NP;
        int lock = 0;
        int64_t ninner = 0;
        std::vector<int> kh;
        if (so.jmax > 0 && NP > 0) {
            kh.resize((size_t)NP * so.jmax);
            CK(cudaMemcpy(kh.data(), so.P.k_hist, kh.size() * sizeof(int), cudaMemcpyDeviceToHost));
        }
        for (int p = 0; p < NP; ++p) {
            const ProbOut& o = so.pr[p];
            lock = std::max(lock, o.outer + (o.brk ? 1 : 0));
            const int cnt = std::min(o.outer + (o.brk ? 1 : 0), so.jmax);
            int64_t kp = 0;
            for (int q = 0; q < cnt; ++q) kp += kh[(size_t)p * so.jmax + q];
            ninner += kp;
            if (st->inner_steps) st->inner_steps[p] = (int32_t)std::min<int64_t>(kp, INT32_MAX);
            if (st->status) st->status[p] = o.status;
            if (st->outer_iters) st->outer_iters[p] = o.outer;
            if (st->rel_res_true) st->rel_res_true[p] = o.rel_true;
            if (st->rel_res_est) st->rel_res_est[p] = o.rel_est;
        }
        st->lockstep_outer = lock;
        st->total_inner = ninner;
        st->kernel_launches = g_launches - launches0;
        float tms = 0.f;
        cudaEventElapsedTime(&tms, h->ev_t0, h->ev_t1);
        st->t_total_ms = tms;
    }
    return status;
}

int sfgmres_autotune(sfgmres_t h, int32_t nrhs, int32_t m, int32_t s, int32_t k, int32_t* block_rows_out,
                     int32_t* spmv_vector_out, double* step_ms_out) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (nrhs < 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "nrhs must be >= 1");
    int rc = check_params(h, m, s, k);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    // candidate row-block sizes: the default rule's size and a ladder of smaller and larger ones (multiples of 32)
    std::vector<int> cand;
    int maxn = 0;
    for (int q = 0; q < h->nsys; ++q) maxn = std::max(maxn, h->sys_n[q]);
    const int base = (h->nsys == 1) ? single_block_rows(h->n, h->sms, h->prec) : kBatchBlockRows;
    for (int v : {base, base / 2, base / 4, base / 8, 512, 1024, 2048, 4096, 8192}) {
        v = std::min(kBlockRowsMax, std::max(256, (v / 32) * 32));
        if (v > ((maxn + 31) / 32) * 32 && v != base) continue;  // larger than every system: same as smaller ones
        if (std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
    }
    // candidate lanes per row: the default rule's choice, and the sub-warp widths for matrices with long rows
    std::vector<int> vecs = {0};
    if (h->maxlen > 16)
        for (int v : {8, 32}) vecs.push_back(v);  // the inner kernel has 8- and 32-lane variants
    const int save_block = h->block_rows, save_vec = h->vec_opt, save_graph = h->use_graph;
    const int steps = std::min(m, 8);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = INFINITY;
    int best_b = save_block, best_v = save_vec;
    for (int bq : cand) {
        h->block_rows = bq;
        set_list_geometry(h);
        for (int vv : vecs) {
            h->vec_opt = vv;
            h->vec = vv ? vv : choose_vec(h->nnz, h->n, h->maxlen);
            Plan P;
            Geo* g = nullptr;
            if ((rc = prepare(h, nrhs, steps, s, k, 0, &P, &g))) break;
            // a unit-norm start vector for every problem (the timing does not depend on its values)
            if ((rc = ensure(h, h->bst, (size_t)P.N * 8))) break;
            if ((rc = ensure(h, h->xst, (size_t)P.N * 8))) break;
            double* v0 = (double*)h->bst.p;
            k_fill<<<grid_for(P.N), 256, 0, h->st>>>(P.N, 1.0 / std::sqrt((double)std::max(1, maxn)), v0);
            float tbest = INFINITY;
            for (int rep = 0; rep < 3 && rc == 0; ++rep) {
                cudaEventRecord(e0, h->st);
                rc = run_cycle(h, P, -1, v0, nullptr, 0, 0, (double*)h->xst.p);
                cudaEventRecord(e1, h->st);
                if (cudaStreamSynchronize(h->st) != cudaSuccess) rc = fail(h, SFGMRES_ERR_CUDA, "autotune run failed");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tbest = std::min(tbest, ms);  // the first run is a warm-up
            }
            if (rc) break;
            const double per_step = tbest / steps;
            if (per_step < best) {
                best = per_step;
                best_b = bq;
                best_v = vv;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->use_graph = save_graph;
    if (rc) {  // leave the handle as it was
        h->block_rows = save_block;
        h->vec_opt = save_vec;
        h->vec = save_vec ? save_vec : choose_vec(h->nnz, h->n, h->maxlen);
        set_list_geometry(h);
        return rc;
    }
    h->block_rows = best_b;
    h->vec_opt = best_v;
    h->vec = best_v ? best_v : choose_vec(h->nnz, h->n, h->maxlen);
    set_list_geometry(h);
    if (block_rows_out) *block_rows_out = h->sys_Bq.empty() ? 0 : h->sys_Bq[0];
    if (spmv_vector_out) *spmv_vector_out = h->vec;
    if (step_ms_out) *step_ms_out = best;
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

int sfgmres_update_values(sfgmres_t h, const double* vals) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!vals && h->nnz > 0) return fail(h, SFGMRES_ERR_INVALID_ARG, "vals must not be NULL");
    CK(cudaSetDevice(h->dev));
    if (h->nnz == 0) return SFGMRES_OK;
    CK(cudaMemcpyAsync(h->val, vals, h->nnz * sizeof(double),
                       is_device_ptr(vals) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    ++h->vals_ver;  // the ILU(0) factors (if any) are recomputed at their next use
    if (h->val32) k_to_f32<<<grid_for(h->nnz), 256, 0, h->st>>>(h->nnz, h->val, h->val32);
    if (h->rpT) {
        launch_gather_vals(h->nnz, h->srcT, h->val, h->valT, h->st);
        if (h->val32T) k_to_f32<<<grid_for(h->nnz), 256, 0, h->st>>>(h->nnz, h->valT, h->val32T);
    }
    for (int t = 0; t < 2; ++t) {  // the length-binned copies' values
        sfgmres_ctx::BCopy& B = h->bc[t];
        if (B.rp && B.ver == h->geo_ver && h->perm[t])
            launch_bcopy_fill(h->nl, t ? h->rpT : h->rp, nullptr, t ? h->valT : h->val, h->lb, h->lb + h->nl,
                              h->perm[t], B.rp, nullptr, B.val, h->st);
        else
            B.ver = -1;  // rebuilt at the next use
    }
    for (int t = 0; t < 2; ++t) {  // the SELL-32 copies' values
        sfgmres_ctx::Sell& S = h->sell[t];
        if (!S.off) continue;
        launch_sell_fill(h->sl_ns, h->sl_sys, h->nsys, h->sl_sys + h->nsys + 1, t ? h->rpT : h->rp, nullptr,
                         t ? h->valT : h->val, S.off, S.len, nullptr, S.val, h->st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    return SFGMRES_OK;
}

int sfgmres_pattern_outer(sfgmres_t h, const double* u, const double* v, double alpha, double* out) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!u || !v || (!out && h->nnz > 0)) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    CK(cudaSetDevice(h->dev));
    launch_pattern_outer(h->n, h->rp, h->col, u, v, alpha, out, h->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    return SFGMRES_OK;
}

int sfgmres_inner_cycle(sfgmres_t h, const double* v, double* z, int32_t m, int32_t s, int32_t k, double* basis,
                        double* y, int32_t* k_out, int32_t* reason_out) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!v || !z || !k_out) return fail(h, SFGMRES_ERR_INVALID_ARG, "v, z and k_out must not be NULL");
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sfgmres_inner_cycle needs a single-system handle");
    int rc = check_params(h, m, s, k);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    Plan P;
    if ((rc = prepare(h, 1, m, s, k, 0, &P, nullptr))) return rc;
    if ((rc = run_cycle(h, P, -1, v, nullptr, 0, 0, z))) return rc;
    CycleState* hc = (CycleState*)h->h_cyc.p;
    CK(cudaMemcpyAsync(hc, P.cyc, sizeof(CycleState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    const CycleState cs = *hc;
    if (P.gsync) {
        unsigned long long gave_up = 0;
        CK(cudaMemcpy(&gave_up, P.gsync + 1, sizeof(gave_up), cudaMemcpyDeviceToHost));
        if (gave_up) return fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
    }
    *k_out = cs.k;
    if (reason_out) *reason_out = cs.reason;
    if (cs.reason == 6) return fail(h, SFGMRES_ERR_NAN, "non-finite value in the inner cycle");
    if (basis) {
        const int cnt = std::min(cs.k + 1, m + 1);
        // vectors formed: k, plus the dropped one after C2; a vector beyond the last SpMV is not formed
        const int formed = (cs.reason == 2) ? cs.k + 1 : cs.k;
        launch_export_basis(P, basis, std::min(cnt, std::max(formed, 1)));
    }
    if (y && cs.k > 0) CK(cudaMemcpyAsync(y, P.y, cs.k * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return cs.k == 0 ? SFGMRES_BREAKDOWN : SFGMRES_OK;
}

int sfgmres_solve_restarted(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                            int32_t k, double tol, int32_t max_cycles, double* res_hist, int32_t* cycles_out) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sfgmres_solve_restarted needs a single-system handle");
    if (max_cycles < 0) return fail(h, SFGMRES_ERR_INVALID_ARG, "max_cycles must be >= 0");
    int rc = check_solve_args(h, b, x, m, s, k, tol);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    Plan P;
    // one outer slot: Vb holds r, nu its scale 1/||r||, Z the cycle's z (nothing else of the outer state is used)
    if ((rc = prepare(h, 1, m, s, k, 1, &P, nullptr))) return rc;
    const size_t nbytes = (size_t)P.N * sizeof(double);
    if ((rc = ensure(h, h->bst, nbytes))) return rc;
    if ((rc = ensure(h, h->xst, nbytes))) return rc;
    double* db = (double*)h->bst.p;
    double* dx = (double*)h->xst.p;
    double* dz = P.Z;
    CK(cudaMemcpyAsync(db, b, nbytes, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (x0) {
        CK(cudaMemcpyAsync(dx, x0, nbytes, is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           h->st));
    } else {
        k_fill<<<grid_for(P.N), 256, 0, h->st>>>(P.N, 0.0, dx);
        ++g_launches;
    }
    OuterState* host_ost = (OuterState*)h->h_ost.p;
    CycleState* hc = (CycleState*)h->h_cyc.p;
    int status = SFGMRES_NOT_CONVERGED, c = 0;
    std::string msg;
    for (;; ++c) {
        // r_c = b - A x_c into the outer slot, beta = ||r_c||, ||b||, nu = 1/beta
        launch_residual(P, db, dx, P.Vb, false);
        launch_init_state(P, tol);
        CK(cudaMemcpyAsync(host_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        CK(cudaGetLastError());
        const OuterState os = host_ost[0];
        if (!std::isfinite(os.beta) || !std::isfinite(os.bnorm) || os.nan) {
            status = SFGMRES_ERR_NAN;
            msg = "non-finite value in the residual";
            break;
        }
        if (res_hist) res_hist[c] = (os.bnorm > 0.0) ? os.beta / os.bnorm : 0.0;
        if (os.beta <= os.tol_abs) {
            status = SFGMRES_OK;
            break;
        }
        if (c == max_cycles) break;
        // z_c: one sGMRES cycle (rules C1, C2) on r_c / beta; x_{c+1} = x_c + beta z_c
        if ((rc = run_cycle(h, P, -1, P.Vb, P.nu, P.jmax + 1, 0, dz))) return rc;
        CK(cudaMemcpyAsync(hc, P.cyc, sizeof(CycleState), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        CK(cudaGetLastError());
        if (P.gsync) {
            unsigned long long gave_up = 0;
            CK(cudaMemcpy(&gave_up, P.gsync + 1, sizeof(gave_up), cudaMemcpyDeviceToHost));
            if (gave_up) return fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
        }
        if (hc->reason == 6) {
            status = SFGMRES_ERR_NAN;
            msg = "non-finite value in the inner cycle";
            break;
        }
        if (hc->k == 0) {  // the cycle accepted no column: x stays
            status = SFGMRES_BREAKDOWN;
            break;
        }
        k_axpy_scalar<<<grid_for(P.N), 256, 0, h->st>>>(P.N, os.beta, dz, dx);
        ++g_launches;
    }
    CK(cudaMemcpyAsync(x, dx, nbytes, is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (cycles_out) *cycles_out = c;
    if (status == SFGMRES_ERR_NAN) return fail(h, SFGMRES_ERR_NAN, msg);
    return status;
}

}  // extern "C"

// ---- multi-level FGMRES (Section 5) ----
namespace {
constexpr int kMaxLowerLevels = 4;

// Write one int of device memory on the handle's stream (a level's per-problem flag word).
int set_flag(sfgmres_ctx* h, const int* flag, int v) {
    CK(cudaMemcpyAsync((void*)flag, &v, sizeof(int), cudaMemcpyHostToDevice, h->st));
    return 0;
}

// The plan of lower level L (1-based) for a basis of at most J steps: the top plan P0 with every outer FGMRES pointer
// replaced by level L's own workspace and flag word.  The inner-cycle workspaces, sketch lists and row blocks are
// shared: the levels run strictly nested, one at a time.
int level_plan(sfgmres_ctx* h, const Plan& P0, int L, int J, Plan* out) {
    if ((int)h->lvl.size() < L) h->lvl.resize(L);
    auto& W = h->lvl[L - 1];
    const size_t N = (size_t)P0.N, nb = (size_t)P0.nblk, Jz = (size_t)J;
    int rc;
    const std::pair<DevBuf*, size_t> need[] = {
        {&W.Vb, (Jz + 1) * N * 8}, {&W.Z, Jz * N * 8},       {&W.nu, (Jz + 1) * 8},     {&W.Wo, N * 8},
        {&W.opart, nb * (Jz + 1) * 8}, {&W.npart, nb * 8}, {&W.npart2, nb * 8},     {&W.h1, (Jz + 1) * 8},
        {&W.h2, (Jz + 1) * 8},     {&W.H, (Jz + 1) * Jz * 8}, {&W.cs, Jz * 8},        {&W.sn, Jz * 8},
        {&W.g, (Jz + 1) * 8},      {&W.yo, Jz * 8},           {&W.est_hist, Jz * 8},  {&W.ffom_hist, Jz * 8},
        {&W.ires_hist, Jz * 8},    {&W.rho_hist, Jz * 8},     {&W.k_hist, Jz * 4},    {&W.reason_hist, Jz * 4},
        {&W.ost, sizeof(OuterState)}, {&W.pflag, sizeof(int)}, {&W.rhs, N * 8}};
    for (const auto& q : need)
        if ((rc = ensure(h, *q.first, q.second))) return rc;
    Plan P = P0;
    P.jmax = J;
    P.Vb = (double*)W.Vb.p;
    P.Z = (double*)W.Z.p;
    P.nu = (double*)W.nu.p;
    P.Wo = (double*)W.Wo.p;
    P.opart = (double*)W.opart.p;
    P.npart = (double*)W.npart.p;
    P.npart2 = (double*)W.npart2.p;
    P.h1 = (double*)W.h1.p;
    P.h2 = (double*)W.h2.p;
    P.H = (double*)W.H.p;
    P.cs = (double*)W.cs.p;
    P.sn = (double*)W.sn.p;
    P.g = (double*)W.g.p;
    P.yo = (double*)W.yo.p;
    P.est_hist = (double*)W.est_hist.p;
    P.ffom_hist = (double*)W.ffom_hist.p;
    P.ires_hist = (double*)W.ires_hist.p;
    P.rho_hist = (double*)W.rho_hist.p;
    P.k_hist = (int*)W.k_hist.p;
    P.reason_hist = (int*)W.reason_hist.p;
    P.ost = (OuterState*)W.ost.p;
    P.pflag = (const int*)W.pflag.p;
    if ((rc = set_flag(h, P.pflag, 0))) return rc;
    *out = P;
    return 0;
}

// Outcome of one run of a lower level.
struct LevelRun {
    int outer = 0;          // outer steps taken
    int reason = 1;         // 3: met its tolerance, 1: used its budget
    double est = INFINITY;  // last Givens estimate relative to the norm of its right-hand side
    int64_t inner = 0;      // sGMRES steps of the lowest-level cycles under this run
    int error = 0;          // SFGMRES_ERR_NAN or SFGMRES_ERR_CUDA
};

// Tolerance the Eq. 5 bound asks of the preconditioner of a level's next step: its target tol_abs over its FFOM
// residual of the previous step (beta before the first), relative to the unit right-hand side v_j; 0 (the child's
// whole budget) with rule C3 off or an undefined FFOM residual.
double child_tolerance(const sfgmres_ctx* h, const OuterState& os, int j) {
    const double fprev = (j == 0) ? os.beta : os.ffom;
    return (h->c3 && std::isfinite(fprev) && fprev > 0.0) ? os.tol_abs / fprev : 0.0;
}

// Lower level L: FGMRES on A z = scale[0] v (zero initial guess) until its Givens estimate meets the relative
// tolerance tau or it has taken its J steps (at least one step either way); its preconditioner is level L + 1, or an
// sGMRES cycle at the lowest level.  The last iterate is written to out (zero if the first step had no correction).
int run_level(sfgmres_ctx* h, const std::vector<Plan>& Ps, int L, const double* v, const double* scale, double tau,
              double* out, LevelRun* res) {
    const Plan& P = Ps[L];
    const int N = P.N, J = P.jmax;
    const bool lowest = (L + 1 == (int)Ps.size());
    OuterState* host_ost = (OuterState*)h->h_ost.p;
    double* rhs = (double*)h->lvl[L - 1].rhs.p;
    k_scale_copy<<<grid_for(N), 256, 0, h->st>>>(N, v, scale, rhs);
    ++g_launches;
    launch_residual(P, rhs, nullptr, P.Vb, false);
    launch_init_state(P, tau);
    CK(cudaMemcpyAsync(host_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    OuterState os = host_ost[0];
    if (!std::isfinite(os.beta) || os.nan) {
        res->error = SFGMRES_ERR_NAN;
        return 0;
    }
    for (int j = 0; j < J; ++j) {
        double* zj = P.Z + (int64_t)j * N;
        if (lowest) {
            int rc = run_cycle(h, P, j, P.Vb + (int64_t)j * N, P.nu + j, J + 1, h->c3, zj);
            if (rc) return rc;
        } else {
            LevelRun cr;
            int rc = run_level(h, Ps, L + 1, P.Vb + (int64_t)j * N, P.nu + j, child_tolerance(h, os, j), zj, &cr);
            if (rc) return rc;
            res->inner += cr.inner;
            if (cr.error) {
                res->error = cr.error;
                return 0;
            }
            k_set_cycle<<<1, 1, 0, h->st>>>(P.cyc, cr.outer, cr.reason, cr.est);
            ++g_launches;
        }
        launch_outer_step(P, j);
        CK(cudaMemcpyAsync(host_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        CK(cudaGetLastError());
        os = host_ost[0];
        if (os.nan) {
            res->error = os.sync_fail ? SFGMRES_ERR_CUDA : SFGMRES_ERR_NAN;
            return 0;
        }
        if (os.breakdown == 2) break;  // step j made no correction: the iterate of step j - 1 stands
        res->outer = j + 1;
        res->est = os.est / os.bnorm;
        if (os.conv_est || os.breakdown == 1) {
            res->reason = 3;
            break;
        }
    }
    if (lowest && res->outer > 0) {
        std::vector<int> kh(res->outer);
        CK(cudaMemcpy(kh.data(), P.k_hist, kh.size() * sizeof(int), cudaMemcpyDeviceToHost));
        for (int q : kh) res->inner += q;
    }
    if (res->outer == 0) {
        k_fill<<<grid_for(N), 256, 0, h->st>>>(N, 0.0, out);
        ++g_launches;
        return 0;
    }
    int rc;
    if ((rc = set_flag(h, P.pflag, 2))) return rc;  // finalise this level's only problem: out = Z y
    launch_final_x(P, J, nullptr, out);
    return set_flag(h, P.pflag, 0);
}

}  // namespace

extern "C" {

int sfgmres_solve_multilevel(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                             int32_t k, double tol, int32_t nlower, const int32_t* level_steps,
                             sfgmres_stats* st) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sfgmres_solve_multilevel needs a single-system handle");
    if (nlower < 1 || nlower > kMaxLowerLevels || !level_steps)
        return fail(h, SFGMRES_ERR_INVALID_ARG, "need 1 <= nlower <= 4 lower levels and their step budgets");
    for (int L = 0; L < nlower; ++L)
        if (level_steps[L] < 1 || level_steps[L] > kMaxM)
            return fail(h, SFGMRES_ERR_INVALID_ARG, "every lower level's budget must be in [1, 1024]");
    int rc = check_solve_args(h, b, x, m, s, k, tol);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int64_t launches0 = g_launches;
    const int jmax = h->max_outer;
    std::vector<Plan> Ps(nlower + 1);
    if ((rc = prepare(h, 1, m, s, k, jmax, &Ps[0], nullptr))) return rc;
    const Plan& P0 = Ps[0];
    for (int L = 1; L <= nlower; ++L)
        if ((rc = level_plan(h, P0, L, level_steps[L - 1], &Ps[L]))) return rc;
    const int N = P0.N;
    const size_t nbytes = (size_t)N * sizeof(double);
    if ((rc = ensure(h, h->bst, nbytes))) return rc;
    if ((rc = ensure(h, h->xst, nbytes))) return rc;
    if ((rc = ensure(h, h->x0st, nbytes))) return rc;
    double* db = (double*)h->bst.p;
    double* dx = (double*)h->xst.p;
    double* dx0 = (double*)h->x0st.p;
    CK(cudaEventRecord(h->ev_t0, h->st));
    CK(cudaMemcpyAsync(db, b, nbytes, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (x0) {
        CK(cudaMemcpyAsync(dx0, x0, nbytes, is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           h->st));
        k_copy<<<grid_for(N), 256, 0, h->st>>>(N, dx0, dx);
    } else {
        k_fill<<<grid_for(N), 256, 0, h->st>>>(N, 0.0, dx);
    }
    ++g_launches;
    const double* px0 = x0 ? dx0 : nullptr;
    OuterState* host_ost = (OuterState*)h->h_ost.p;
    launch_residual(P0, db, px0, P0.Vb, false);
    launch_init_state(P0, tol);
    CK(cudaMemcpyAsync(host_ost, P0.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    OuterState os = host_ost[0];
    int status = SFGMRES_NOT_CONVERGED, outer = 0;
    double rel_true = 0.0, rel_est = 0.0;
    int64_t total_inner = 0;
    std::string msg;
    bool done = false;
    if (!std::isfinite(os.beta) || !std::isfinite(os.bnorm) || os.nan) {
        return fail(h, SFGMRES_ERR_NAN, "non-finite value in b or x0 (or in A x0)");
    } else if (os.bnorm == 0.0) {  // x = 0
        k_fill<<<grid_for(N), 256, 0, h->st>>>(N, 0.0, dx);
        ++g_launches;
        status = SFGMRES_OK;
        done = true;
    } else if (os.beta <= os.tol_abs) {  // x0 already meets the tolerance
        status = SFGMRES_OK;
        rel_true = rel_est = os.beta / os.bnorm;
        done = true;
    }
    for (int j = 0; j < jmax && !done; ++j) {
        LevelRun cr;
        if ((rc = run_level(h, Ps, 1, P0.Vb + (int64_t)j * N, P0.nu + j, child_tolerance(h, os, j),
                            P0.Z + (int64_t)j * N, &cr)))
            return rc;
        total_inner += cr.inner;
        if (cr.error == SFGMRES_ERR_CUDA) return fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
        if (cr.error) return fail(h, SFGMRES_ERR_NAN, "non-finite value during the iteration");
        k_set_cycle<<<1, 1, 0, h->st>>>(P0.cyc, cr.outer, cr.reason, cr.est);
        ++g_launches;
        launch_outer_step(P0, j);
        CK(cudaMemcpyAsync(host_ost, P0.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        CK(cudaGetLastError());
        os = host_ost[0];
        if (os.nan) {
            if (os.sync_fail) return fail(h, SFGMRES_ERR_CUDA, "the fused inner step's grid-wide wait gave up");
            return fail(h, SFGMRES_ERR_NAN, "non-finite value during the iteration");
        }
        const bool brk = (os.breakdown == 2);
        const bool last = (j + 1 == jmax);
        if (!brk) {
            outer = j + 1;
            rel_est = os.est / os.bnorm;
        }
        if (brk || os.conv_est || os.breakdown == 1 || last) {
            // x = x0 + Z y over the steps taken, and its recomputed residual
            if ((rc = set_flag(h, P0.pflag, 2))) return rc;
            launch_final_x(P0, jmax, px0, dx);
            launch_residual(P0, db, dx, nullptr, true);
            launch_true_residual_reduce(P0);
            CK(cudaMemcpyAsync(host_ost, P0.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            CK(cudaGetLastError());
            if ((rc = set_flag(h, P0.pflag, 0))) return rc;
            os = host_ost[0];
            rel_true = std::sqrt(os.true_res2) / os.bnorm;
            if (brk) status = SFGMRES_BREAKDOWN;
            else if (rel_true <= tol || os.breakdown == 1) status = SFGMRES_OK;
            else if (last) status = SFGMRES_NOT_CONVERGED;
            else continue;
            done = true;
        }
    }
    CK(cudaMemcpyAsync(x, dx, nbytes, is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaEventRecord(h->ev_t1, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (st) {
        st->status = status;
        st->outer_iters = outer;
        st->total_inner = (int32_t)std::min<int64_t>(total_inner, INT32_MAX);
        st->rel_res_true = rel_true;
        st->rel_res_est = rel_est;
        const int cnt = std::min(outer + (status == SFGMRES_BREAKDOWN ? 1 : 0), jmax);
        const int cap = std::min(cnt, st->hist_cap);
        if (cap > 0) {
            std::vector<int> kh(cap), rh(cap);
            std::vector<double> eh(cap), fh(cap), ih(cap), qh(cap);
            CK(cudaMemcpy(kh.data(), P0.k_hist, cap * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(rh.data(), P0.reason_hist, cap * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(eh.data(), P0.est_hist, cap * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fh.data(), P0.ffom_hist, cap * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(ih.data(), P0.ires_hist, cap * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(qh.data(), P0.rho_hist, cap * sizeof(double), cudaMemcpyDeviceToHost));
            for (int q = 0; q < cap; ++q) {
                if (st->inner_k) st->inner_k[q] = kh[q];
                if (st->inner_reason) st->inner_reason[q] = rh[q];
                if (st->res_est && q < outer) st->res_est[q] = eh[q];
                if (st->ffom_res && q < outer) st->ffom_res[q] = fh[q];
                if (st->inner_res && q < outer) st->inner_res[q] = ih[q];
                if (st->inner_rho && q < outer) st->inner_rho[q] = qh[q];
            }
        }
        st->kernel_launches = g_launches - launches0;
        float tms = 0.f;
        cudaEventElapsedTime(&tms, h->ev_t0, h->ev_t1);
        st->t_total_ms = tms;
        st->t_inner_spmv_ms = st->t_inner_axpy_ms = st->t_qr_ms = 0.0;
        st->n_inner_spmv = st->n_inner_axpy = st->n_qr = 0;
        st->t_step_span_ms = 0.0;
        st->n_step_span = 0;
    }
    return status;
}

int sfgmres_precond_info(sfgmres_t h, int32_t* colour, int32_t* ncolours, double* lu) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    CK(cudaSetDevice(h->dev));
    int rc = ensure_ilu(h);
    if (rc) return rc;
    if (colour) std::memcpy(colour, h->ilu_colour.data(), (size_t)h->n * sizeof(int32_t));
    if (ncolours) *ncolours = h->ilu.ncol;
    if (lu && h->nnz > 0) {
        std::vector<double> v((size_t)h->nnz);
        CK(cudaMemcpy(v.data(), h->ilu_lu.p, (size_t)h->nnz * sizeof(double), cudaMemcpyDeviceToHost));
        for (int64_t p = 0; p < h->nnz; ++p) lu[h->ilu_src[p]] = v[p];
    }
    return SFGMRES_OK;
}

int sfgmres_sketch_apply(sfgmres_t h, int32_t s, const double* v, double* c) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!v || !c) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sfgmres_sketch_apply needs a single-system handle");
    int rc = check_params(h, 1, s, 0);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    Plan P;
    const int save = h->prec;
    h->prec = kFP64;
    rc = prepare(h, 1, 1, s, 0, 0, &P, nullptr);
    h->prec = save;
    if (rc) return rc;
    launch_sketch_partials(P, v, nullptr, 0, nullptr, P.cpart);
    launch_sketch_reduce(P, P.cpart, c, nullptr);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

int sfgmres_sketch_pattern(sfgmres_t h, int32_t s, int32_t* rows, int8_t* signs) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!rows || !signs) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    if (h->nsys != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "sfgmres_sketch_pattern needs a single-system handle");
    int rc = check_params(h, 1, s, 0);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int zeta = (h->kind == 1) ? 1 : h->zeta;
    int8_t* neg = nullptr;
    CK(cudaMalloc(&neg, (size_t)h->n * zeta));
    launch_sketch_pattern(h->n, s, zeta, h->kind, h->seed, rows, neg, h->st);
    const int64_t cnt = (int64_t)h->n * zeta;
    k_neg_to_sign<<<grid_for(cnt), 256, 0, h->st>>>(cnt, neg, signs);
    ++g_launches;
    cudaError_t e1 = cudaStreamSynchronize(h->st);
    cudaFree(neg);
    CK(e1);
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

int sfgmres_spmv(sfgmres_t h, const double* xv, double* yv) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!xv || !yv) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    CK(cudaSetDevice(h->dev));
    Geo* g = nullptr;
    int rc = get_geometry(h, 1, &g);
    if (rc) return rc;
    if (h->vec == 0 && (rc = ensure_bins(h, false))) return rc;
    Plan P;
    plan_geometry(h, g, false, P);
    launch_spmv_f64(P, xv, yv);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

}  // extern "C"
