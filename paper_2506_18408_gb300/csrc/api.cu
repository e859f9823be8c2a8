// C ABI of the sketched-FGMRES library: handle management, validation, workspaces and the host-side driver loop.
//
// The driver enqueues every step on the handle's stream; the device state (CycleState / OuterState) carries the
// decisions of the stop rules, so the host synchronises once per outer FGMRES step to read the convergence flags.
#include "../../include/sfgmres.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace sfg;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace

namespace sfg {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace sfg

struct sfgmres_ctx {
    int dev = 0;
    int n = 0;
    int64_t nnz = 0;
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
    uint64_t seed = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t qst = nullptr;       // side stream of the sketched-QR cluster kernel
    cudaEvent_t ev_c = nullptr;       // "sketched column ready" (main -> side)
    cudaEvent_t ev_q = nullptr;       // "cycle's QR updates done" (side -> main)
    int sms = 152;
    int maxlen = 0;                   // longest CSR row

    // options
    int prec = kFP64, zeta = 8, c3 = 1, max_outer = 50, kind = 0, profile = 0, vec_opt = 0;
    double cond_thr = 1e15;

    // geometry
    int Bn = 0, nblk = 0, vec = 8;

    // sketch gather lists (cached for one (s, zeta, kind))
    int sk_s = -1, sk_zeta = -1, sk_kind = -1, sk_headroom = 0;
    int* seg = nullptr;
    uint16_t* ent = nullptr;

    // workspaces
    DevBuf U, W, sigma, normpart, hpart, cpart, C, Q, R, d, e, c0, rho, y, coef, hco, cyc;
    DevBuf Vb, Z, nu, Wo, opart, npart, npart2, h1, h2, H, cs, sn, g, yo, est_hist, ffom_hist, k_hist, reason_hist,
        ost;
    DevBuf bst, xst, x0st;  // staging / internal copies

    // pinned host mirrors of the device state
    OuterState* h_ost = nullptr;
    CycleState* h_cyc = nullptr;

    // profiling
    std::vector<EventPair> ev_spmv, ev_axpy, ev_qr;
    size_t n_spmv = 0, n_axpy = 0, n_qr = 0;
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

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
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

// Lanes per CSR row: one thread per row when every row is short (stencils), else a sub-warp sized by the mean.
int choose_vec(int64_t nnz, int n, int maxlen) {
    if (maxlen <= 16) return 1;
    const double avg = n ? (double)nnz / n : 1.0;
    if (avg <= 3.0) return 2;
    if (avg <= 6.0) return 4;
    if (avg <= 12.0) return 8;
    if (avg <= 24.0) return 16;
    return 32;
}

// Row blocks: nblk a multiple of the SM count where possible, Bn a multiple of 32 and <= kBlockRowsMax.
void choose_blocks(int n, int sms, int* Bn, int* nblk) {
    int q = 1, b = 32;
    for (;;) {
        const int64_t per = ((int64_t)n + (int64_t)sms * q - 1) / ((int64_t)sms * q);
        b = (int)(((per + 31) / 32) * 32);
        if (b <= kBlockRowsMax) break;
        q *= 2;
    }
    b = std::max(b, 32);
    *Bn = b;
    *nblk = (int)(((int64_t)n + b - 1) / b);
}

// ---- CSR validation on the device ----
__global__ void k_validate_csr(int n, int64_t nnz, const int64_t* __restrict__ rp64, const int* __restrict__ col,
                               int* __restrict__ rp32, int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) {
        const int64_t v = rp64[i];
        if (v < 0 || v > nnz) atomicOr(bad, 1);
        if (i == 0 && v != 0) atomicOr(bad, 2);
        if (i == n && v != nnz) atomicOr(bad, 4);
        if (i < n && rp64[i + 1] < v) atomicOr(bad, 8);
        if (i < n) {
            const int64_t len = rp64[i + 1] - v;
            if (len > 0) atomicMax(bad + 1, (int)min(len, (int64_t)INT32_MAX));
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

__global__ void k_copy(int n, const double* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_fill(int n, double v, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = v;
}

__global__ void k_neg_to_sign(int64_t cnt, const int8_t* __restrict__ a, int8_t* __restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = a[i] ? (int8_t)-1 : (int8_t)1;
}

int grid_for(int64_t n, int th = 256) { return (int)std::min<int64_t>((n + th - 1) / th, 152 * 16); }

int build_sketch(sfgmres_ctx* h, int s) {
    const int zeta = (h->kind == 1) ? 1 : h->zeta;
    if (h->seg && h->sk_s == s && h->sk_zeta == zeta && h->sk_kind == h->kind) return 0;
    if (h->seg) cudaFree(h->seg);
    if (h->ent) cudaFree(h->ent);
    h->seg = nullptr;
    h->ent = nullptr;
    h->sk_s = -1;
    const int64_t tot = (int64_t)h->n * zeta;
    const int64_t nseg = (int64_t)h->nblk * s + 1;
    if (nseg > INT32_MAX || tot + 8 * nseg >= INT32_MAX)
        return fail(h, SFGMRES_ERR_INVALID_ARG, "sketch too large for 32-bit gather lists");
    int* rows = nullptr;
    int8_t* neg = nullptr;
    int* counts = nullptr;
    CK(cudaMalloc(&rows, tot * sizeof(int)));
    CK(cudaMalloc(&neg, tot));
    CK(cudaMalloc(&counts, nseg * sizeof(int)));
    CK(cudaMalloc(&h->seg, nseg * sizeof(int)));
    CK(cudaMemsetAsync(counts, 0, nseg * sizeof(int), h->st));
    Plan dummy;
    launch_sketch_pattern(dummy, h->n, s, zeta, h->kind, h->seed, rows, neg, h->st);
    launch_sketch_count(h->n, s, zeta, h->Bn, h->nblk, rows, counts, h->seg, h->st);
    std::vector<int> hs(nseg);
    CK(cudaMemcpyAsync(hs.data(), h->seg, nseg * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const int64_t total = hs[nseg - 1];
    CK(cudaMalloc(&h->ent, (total + 8) * sizeof(uint16_t)));  // +8: room for one padding group
    launch_sketch_fill(h->n, s, zeta, h->Bn, h->nblk, rows, neg, h->seg, h->ent, total, h->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    cudaFree(rows);
    cudaFree(neg);
    cudaFree(counts);
    {
        // FP64 sketch terms are 53-bit integers summed exactly in 64 bits: lists longer than 1023 entries get
        // extra right shifts so that no sum can overflow
        int longest = 0;
        for (int64_t q = 0; q + 1 < nseg; ++q) longest = std::max(longest, hs[q + 1] - hs[q]);
        int H = 0;
        while ((longest >> H) >= 1023) ++H;
        h->sk_headroom = H;
    }
    h->sk_s = s;
    h->sk_zeta = zeta;
    h->sk_kind = h->kind;
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

// A^T in CSR form, built on first use (deterministic layout) and kept; values follow sfgmres_update_values.
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

// Allocates the workspaces of a solve and fills a Plan (for A, or for A^T when transpose is set).
int prepare(sfgmres_ctx* h, int m, int s, int t, int jmax, Plan* p, bool transpose = false) {
    int rc;
    if ((rc = build_sketch(h, s))) return rc;
    if (transpose && (rc = ensure_transpose(h))) return rc;
    if (h->prec != kFP64 && (rc = ensure_f32(h, transpose))) return rc;
    const size_t vt = (h->prec == kFP64) ? 8 : (h->prec == kFP32 ? 4 : 2);
    const size_t at = (h->prec == kFP64) ? 8 : 4;
    const size_t n = (size_t)h->n;
    const size_t nb = (size_t)h->nblk;
    if ((rc = ensure(h, h->U, (size_t)(m + 1) * n * vt))) return rc;
    if ((rc = ensure(h, h->W, n * at))) return rc;
    if ((rc = ensure(h, h->sigma, (m + 1) * 8))) return rc;
    if ((rc = ensure(h, h->normpart, 2 * nb * at))) return rc;
    if ((rc = ensure(h, h->hpart, nb * kMaxTrunc * at))) return rc;
    if ((rc = ensure(h, h->cpart, nb * s * at))) return rc;
    if ((rc = ensure(h, h->C, (size_t)m * s * 8))) return rc;
    if ((rc = ensure(h, h->Q, (size_t)m * s * 8))) return rc;
    if ((rc = ensure(h, h->R, (size_t)m * m * 8))) return rc;
    if ((rc = ensure(h, h->d, m * 8))) return rc;
    if ((rc = ensure(h, h->e, s * 8))) return rc;
    if ((rc = ensure(h, h->c0, s * 8))) return rc;
    if ((rc = ensure(h, h->rho, m * 8))) return rc;
    if ((rc = ensure(h, h->y, m * 8))) return rc;
    if ((rc = ensure(h, h->coef, m * 8))) return rc;
    if ((rc = ensure(h, h->hco, (size_t)m * kMaxTrunc * 8))) return rc;
    if ((rc = ensure(h, h->cyc, sizeof(CycleState)))) return rc;
    if (jmax > 0) {
        const size_t J = (size_t)jmax;
        if ((rc = ensure(h, h->Vb, (J + 1) * n * 8))) return rc;
        if ((rc = ensure(h, h->Z, J * n * 8))) return rc;
        if ((rc = ensure(h, h->nu, (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->Wo, n * 8))) return rc;
        if ((rc = ensure(h, h->opart, nb * (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->h1, (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->h2, (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->H, (J + 1) * J * 8))) return rc;
        if ((rc = ensure(h, h->cs, J * 8))) return rc;
        if ((rc = ensure(h, h->sn, J * 8))) return rc;
        if ((rc = ensure(h, h->g, (J + 1) * 8))) return rc;
        if ((rc = ensure(h, h->yo, J * 8))) return rc;
        if ((rc = ensure(h, h->est_hist, J * 8))) return rc;
        if ((rc = ensure(h, h->ffom_hist, J * 8))) return rc;
        if ((rc = ensure(h, h->k_hist, J * 4))) return rc;
        if ((rc = ensure(h, h->reason_hist, J * 4))) return rc;
    }
    if ((rc = ensure(h, h->npart, nb * 8))) return rc;
    if ((rc = ensure(h, h->npart2, nb * 8))) return rc;
    if ((rc = ensure(h, h->ost, sizeof(OuterState)))) return rc;

    Plan& P = *p;
    P.n = h->n;
    P.nnz = h->nnz;
    P.rp = transpose ? h->rpT : h->rp;
    P.col = transpose ? h->colT : h->col;
    P.val = transpose ? h->valT : h->val;
    P.val32 = transpose ? h->val32T : h->val32;
    P.vec = transpose ? (h->vec_opt ? h->vec_opt : h->vecT) : h->vec;
    P.Bn = h->Bn;
    P.nblk = h->nblk;
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
    P.R = (double*)h->R.p;
    P.d = (double*)h->d.p;
    P.e = (double*)h->e.p;
    P.c0 = (double*)h->c0.p;
    P.rho = (double*)h->rho.p;
    P.y = (double*)h->y.p;
    P.coef = (double*)h->coef.p;
    P.hco = (double*)h->hco.p;
    P.cyc = (CycleState*)h->cyc.p;
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
    P.k_hist = (int*)h->k_hist.p;
    P.reason_hist = (int*)h->reason_hist.p;
    P.ost = (OuterState*)h->ost.p;
    P.st = h->st;
    return 0;
}

int check_params(sfgmres_ctx* h, int m, int s, int t) {
    if (m < 1 || m > kMaxM) return fail(h, SFGMRES_ERR_INVALID_ARG, "m must be in [1, 1024]");
    if (t < 0 || t > kMaxTrunc) return fail(h, SFGMRES_ERR_INVALID_ARG, "k (truncation) must be in [0, 8]");
    if (h->kind == 1) {
        if (s != h->n) return fail(h, SFGMRES_ERR_INVALID_ARG, "identity sketch needs s == n");
        if (s > kMaxS) return fail(h, SFGMRES_ERR_INVALID_ARG, "identity sketch needs n <= 4096");
    } else {
        if (s < h->zeta || s > kMaxS) return fail(h, SFGMRES_ERR_INVALID_ARG, "s must be in [zeta, 4096]");
    }
    if (m > s) return fail(h, SFGMRES_ERR_INVALID_ARG, "m must not exceed s");
    return 0;
}

// ---- profiling helpers ----
void ev_begin(sfgmres_ctx*, std::vector<EventPair>& pool, size_t idx, cudaStream_t st) {
    if (idx >= pool.size()) {
        EventPair e;
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        pool.push_back(e);
    }
    cudaEventRecord(pool[idx].a, st);
}
void ev_end(sfgmres_ctx*, std::vector<EventPair>& pool, size_t idx, cudaStream_t st) {
    cudaEventRecord(pool[idx].b, st);
}
double ev_sum(const std::vector<EventPair>& pool, size_t count) {
    double tot = 0.0;
    for (size_t i = 0; i < count; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pool[i].a, pool[i].b) == cudaSuccess) tot += ms;
    }
    return tot;
}

// One inner cycle (Section 3) on u_0 = vscale * v; j >= 0 inside a solve (C3 as configured), j < 0 standalone.
// The sketched-QR update of step i runs on the side stream after step i's sketch column is ready, overlapping the
// next step's SpMV; the main stream waits for the last QR update before the least-squares solve.
int run_cycle(sfgmres_ctx* h, const Plan& P, int j, const double* v, const double* vscale, int c3, double* z) {
    launch_cycle_start(P, j, v, vscale, c3, h->cond_thr);
    for (int i = 0; i < P.m; ++i) {
        const bool last = (i == P.m - 1);
        if (h->profile) ev_begin(h, h->ev_spmv, h->n_spmv, h->st);
        launch_inner_spmv(P, i);
        if (h->profile) ev_end(h, h->ev_spmv, h->n_spmv++, h->st);
        if (h->profile) ev_begin(h, h->ev_axpy, h->n_axpy, h->st);
        launch_inner_axpy(P, i, last);
        if (h->profile) ev_end(h, h->ev_axpy, h->n_axpy++, h->st);
        CK(cudaEventRecord(h->ev_c, h->st));
        CK(cudaStreamWaitEvent(h->qst, h->ev_c, 0));
        if (h->profile) ev_begin(h, h->ev_qr, h->n_qr, h->qst);
        CK(launch_inner_qr(P, i, h->qst));
        if (h->profile) ev_end(h, h->ev_qr, h->n_qr++, h->qst);
    }
    CK(cudaEventRecord(h->ev_q, h->qst));
    CK(cudaStreamWaitEvent(h->st, h->ev_q, 0));
    launch_inner_finish(P, z);
    return 0;
}

}  // namespace

// =====================================================================================================================
extern "C" {

const char* sfgmres_version(void) { return "sfgmres-gb300 0.1 (sm_103a)"; }

const char* sfgmres_last_error(sfgmres_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int sfgmres_create(sfgmres_t* out, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* vals, uint64_t sketch_seed, int32_t flags, void* stream) {
    sfgmres_ctx* h = nullptr;
    if (!out) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > INT32_MAX - 1) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "n must be in [1, 2^31-2]");
    if (nnz < 0 || nnz > INT32_MAX) return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "nnz must be in [0, 2^31-1]");
    if (!row_ptr || (nnz > 0 && (!col_idx || !vals)))
        return fail(nullptr, SFGMRES_ERR_INVALID_ARG, "NULL CSR array");
    h = new sfgmres_ctx();
    h->n = (int)n;
    h->nnz = nnz;
    h->seed = sketch_seed;
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
    if (cudaMalloc(&h->rp, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->col, std::max<int64_t>(nnz, 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->val, std::max<int64_t>(nnz, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&rp64, (n + 1) * sizeof(int64_t)) != cudaSuccess || cudaMalloc(&bad, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (rp64) cudaFree(rp64);
        if (bad) cudaFree(bad);
        return bail(SFGMRES_ERR_OOM, "out of device memory for the CSR copy");
    }
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaMemcpyAsync(rp64, row_ptr, (n + 1) * sizeof(int64_t), kind, h->st);
    if (nnz > 0) {
        cudaMemcpyAsync(h->col, col_idx, nnz * sizeof(int), kind, h->st);
        cudaMemcpyAsync(h->val, vals, nnz * sizeof(double), kind, h->st);
    }
    cudaMemsetAsync(bad, 0, 2 * sizeof(int), h->st);
    const int64_t cover = std::max<int64_t>(n + 1, nnz);
    k_validate_csr<<<(int)((cover + 255) / 256), 256, 0, h->st>>>((int)n, nnz, rp64, h->col, h->rp, bad);
    int hbad2[2] = {0, 0};
    cudaMemcpyAsync(hbad2, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st);
    ce = cudaStreamSynchronize(h->st);
    cudaFree(rp64);
    cudaFree(bad);
    if (ce != cudaSuccess) return bail(SFGMRES_ERR_CUDA, std::string("CSR upload: ") + cudaGetErrorString(ce));
    const int hbad = hbad2[0];
    h->maxlen = hbad2[1];
    if (hbad) {
        char buf[160];
        snprintf(buf, sizeof buf, "invalid CSR (code %d: 1 range, 2 row_ptr[0]!=0, 4 row_ptr[n]!=nnz, "
                 "8 decreasing row_ptr, 16 column out of range)", hbad);
        return bail(SFGMRES_ERR_INVALID_ARG, buf);
    }
    choose_blocks(h->n, h->sms, &h->Bn, &h->nblk);
    h->vec = choose_vec(nnz, h->n, h->maxlen);
    if (cudaMallocHost(&h->h_ost, sizeof(OuterState)) != cudaSuccess ||
        cudaMallocHost(&h->h_cyc, sizeof(CycleState)) != cudaSuccess) {
        cudaGetLastError();
        return bail(SFGMRES_ERR_OOM, "cudaMallocHost failed");
    }
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
    DevBuf* bufs[] = {&h->U, &h->W, &h->sigma, &h->normpart, &h->hpart, &h->cpart, &h->C, &h->Q, &h->R, &h->d,
                      &h->e, &h->c0, &h->rho, &h->y, &h->coef, &h->hco, &h->cyc, &h->Vb, &h->Z, &h->nu, &h->Wo,
                      &h->opart, &h->npart, &h->npart2, &h->h1, &h->h2, &h->H, &h->cs, &h->sn, &h->g, &h->yo,
                      &h->est_hist, &h->ffom_hist, &h->k_hist, &h->reason_hist, &h->ost, &h->bst, &h->xst,
                      &h->x0st};
    for (DevBuf* b : bufs) release(*b);
    if (h->h_ost) cudaFreeHost(h->h_ost);
    if (h->h_cyc) cudaFreeHost(h->h_cyc);
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
            h->prec = iv;
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
            if (iv != 0 && iv != 1) return fail(h, SFGMRES_ERR_INVALID_ARG, "profile must be 0 or 1");
            h->profile = iv;
            return 0;
        case SFGMRES_OPT_SPMV_VECTOR:
            if (!(iv == 0 || iv == 2 || iv == 4 || iv == 8 || iv == 16 || iv == 32) || iv != v)
                return fail(h, SFGMRES_ERR_INVALID_ARG, "spmv vector width must be 0, 2, 4, 8, 16 or 32");
            h->vec_opt = iv;
            h->vec = iv ? iv : choose_vec(h->nnz, h->n, h->maxlen);
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
        default: return fail(h, SFGMRES_ERR_INVALID_ARG, "unknown option key");
    }
}

static int solve_impl(sfgmres_t h, bool transpose, const double* b, const double* x0, double* x, int32_t m,
                      int32_t s, int32_t k, double tol, sfgmres_stats* st) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!b || !x) return fail(h, SFGMRES_ERR_INVALID_ARG, "b and x must not be NULL");
    if (!(tol > 0.0 && tol < 1.0)) return fail(h, SFGMRES_ERR_INVALID_ARG, "tol must be in (0, 1)");
    int rc = check_params(h, m, s, k);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int64_t launches0 = g_launches;
    const int jmax = h->max_outer;
    Plan P;
    if ((rc = prepare(h, m, s, k, jmax, &P, transpose))) return rc;
    const size_t nbytes = (size_t)h->n * sizeof(double);
    if ((rc = ensure(h, h->bst, nbytes))) return rc;
    if ((rc = ensure(h, h->xst, nbytes))) return rc;
    if ((rc = ensure(h, h->x0st, nbytes))) return rc;
    double* db = (double*)h->bst.p;
    double* dx = (double*)h->xst.p;
    double* dx0 = (double*)h->x0st.p;
    const bool x_dev = is_device_ptr(x);
    h->n_spmv = h->n_axpy = h->n_qr = 0;
    CK(cudaEventRecord(h->ev_t0, h->st));
    // private copies of b and x0 (x may alias x0, and host inputs are staged)
    CK(cudaMemcpyAsync(db, b, nbytes, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (x0) {
        CK(cudaMemcpyAsync(dx0, x0, nbytes, is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           h->st));
    }
    const double* px0 = x0 ? dx0 : nullptr;
    // r0 = b - A x0 into v_0; beta, ||b||
    launch_residual(P, db, px0, P.Vb);
    launch_init_state(P, tol, jmax);
    CK(cudaMemcpyAsync(h->h_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    OuterState os = *h->h_ost;
    int status = SFGMRES_OK;
    int outer = 0;
    double rel_true = 0.0, rel_est = 0.0;
    bool have_x = false;
    if (!std::isfinite(os.beta) || !std::isfinite(os.bnorm) || os.nan) {
        return fail(h, SFGMRES_ERR_NAN, "non-finite value in b or x0 (or in A x0)");
    }
    if (os.bnorm == 0.0) {  // x = 0
        k_fill<<<grid_for(h->n), 256, 0, h->st>>>(h->n, 0.0, dx);
        ++g_launches;
        have_x = true;
    } else if (os.beta <= os.tol_abs) {  // x0 already meets the tolerance
        if (x0) k_copy<<<grid_for(h->n), 256, 0, h->st>>>(h->n, dx0, dx);
        else k_fill<<<grid_for(h->n), 256, 0, h->st>>>(h->n, 0.0, dx);
        ++g_launches;
        have_x = true;
        rel_true = os.beta / os.bnorm;
        rel_est = rel_true;
    } else {
        status = SFGMRES_NOT_CONVERGED;
        for (int j = 0; j < jmax; ++j) {
            if ((rc = run_cycle(h, P, j, P.Vb + (int64_t)j * h->n, P.nu + j, h->c3, P.Z + (int64_t)j * h->n)))
                return rc;
            launch_outer_step(P, j);
            CK(cudaMemcpyAsync(h->h_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            CK(cudaGetLastError());
            os = *h->h_ost;
            if (os.nan) return fail(h, SFGMRES_ERR_NAN, "non-finite value during the iteration");
            if (os.breakdown == 2) {  // the inner cycle accepted no column: keep the iterate of step j
                status = SFGMRES_BREAKDOWN;
                if (j > 0) {
                    launch_final_x(P, j, px0, dx);
                    launch_residual(P, db, dx, nullptr);
                    launch_true_residual_reduce(P);
                } else {
                    if (x0) k_copy<<<grid_for(h->n), 256, 0, h->st>>>(h->n, dx0, dx);
                    else k_fill<<<grid_for(h->n), 256, 0, h->st>>>(h->n, 0.0, dx);
                    ++g_launches;
                    launch_residual(P, db, px0, nullptr);
                    launch_true_residual_reduce(P);
                }
                outer = j;
                have_x = true;
                break;
            }
            outer = j + 1;
            rel_est = os.est / os.bnorm;
            const bool last = (j + 1 == jmax);
            if (os.conv_est || os.breakdown == 1 || last) {
                launch_final_x(P, j + 1, px0, dx);
                launch_residual(P, db, dx, nullptr);
                launch_true_residual_reduce(P);
                CK(cudaMemcpyAsync(h->h_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
                CK(cudaStreamSynchronize(h->st));
                os = *h->h_ost;
                rel_true = std::sqrt(os.true_res2) / os.bnorm;
                have_x = true;
                if (rel_true <= tol || os.breakdown == 1) {
                    status = SFGMRES_OK;
                    break;
                }
            }
        }
    }
    if (!have_x) return fail(h, SFGMRES_ERR_CUDA, "internal: no iterate formed");
    CK(cudaMemcpyAsync(x, dx, nbytes, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_ost, P.ost, sizeof(OuterState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaEventRecord(h->ev_t1, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (status == SFGMRES_BREAKDOWN) rel_true = std::sqrt(h->h_ost->true_res2) / h->h_ost->bnorm;
    if (st) {
        st->status = status;
        st->outer_iters = outer;
        st->rel_res_true = rel_true;
        st->rel_res_est = rel_est;
        const int cnt = std::min(outer + (status == SFGMRES_BREAKDOWN ? 1 : 0), jmax);
        std::vector<int> kh(std::max(cnt, 1)), rh(std::max(cnt, 1));
        std::vector<double> eh(std::max(cnt, 1)), fh(std::max(cnt, 1));
        if (cnt > 0) {
            CK(cudaMemcpy(kh.data(), P.k_hist, cnt * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(rh.data(), P.reason_hist, cnt * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(eh.data(), P.est_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fh.data(), P.ffom_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
        }
        int tot = 0;
        for (int q = 0; q < cnt; ++q) tot += kh[q];
        st->total_inner = tot;
        const int cap = std::min(cnt, st->hist_cap);
        for (int q = 0; q < cap; ++q) {
            if (st->inner_k) st->inner_k[q] = kh[q];
            if (st->inner_reason) st->inner_reason[q] = rh[q];
            if (st->res_est && q < outer) st->res_est[q] = eh[q];
            if (st->ffom_res && q < outer) st->ffom_res[q] = fh[q];
        }
        st->kernel_launches = g_launches - launches0;
        float tms = 0.f;
        cudaEventElapsedTime(&tms, h->ev_t0, h->ev_t1);
        st->t_total_ms = tms;
        if (h->profile) {
            st->t_inner_spmv_ms = ev_sum(h->ev_spmv, h->n_spmv);
            st->n_inner_spmv = (int64_t)h->n_spmv;
            st->t_inner_axpy_ms = ev_sum(h->ev_axpy, h->n_axpy);
            st->n_inner_axpy = (int64_t)h->n_axpy;
            st->t_qr_ms = ev_sum(h->ev_qr, h->n_qr);
            st->n_qr = (int64_t)h->n_qr;
        } else {
            st->t_inner_spmv_ms = st->t_inner_axpy_ms = st->t_qr_ms = 0.0;
            st->n_inner_spmv = st->n_inner_axpy = st->n_qr = 0;
        }
    }
    return status;
}

int sfgmres_solve(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s, int32_t k,
                  double tol, sfgmres_stats* st) {
    return solve_impl(h, false, b, x0, x, m, s, k, tol, st);
}

int sfgmres_solve_transpose(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                            int32_t k, double tol, sfgmres_stats* st) {
    return solve_impl(h, true, b, x0, x, m, s, k, tol, st);
}

int sfgmres_update_values(sfgmres_t h, const double* vals) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!vals && h->nnz > 0) return fail(h, SFGMRES_ERR_INVALID_ARG, "vals must not be NULL");
    CK(cudaSetDevice(h->dev));
    if (h->nnz == 0) return SFGMRES_OK;
    CK(cudaMemcpyAsync(h->val, vals, h->nnz * sizeof(double),
                       is_device_ptr(vals) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (h->val32) k_to_f32<<<grid_for(h->nnz), 256, 0, h->st>>>(h->nnz, h->val, h->val32);
    if (h->rpT) {
        launch_gather_vals(h->nnz, h->srcT, h->val, h->valT, h->st);
        if (h->val32T) k_to_f32<<<grid_for(h->nnz), 256, 0, h->st>>>(h->nnz, h->valT, h->val32T);
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
    int rc = check_params(h, m, s, k);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    Plan P;
    if ((rc = prepare(h, m, s, k, 0, &P))) return rc;
    if ((rc = run_cycle(h, P, -1, v, nullptr, 0, z))) return rc;
    CK(cudaMemcpyAsync(h->h_cyc, P.cyc, sizeof(CycleState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    const CycleState cs = *h->h_cyc;
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

int sfgmres_sketch_apply(sfgmres_t h, int32_t s, const double* v, double* c) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!v || !c) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    int rc = check_params(h, 1, s, 0);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    if ((rc = build_sketch(h, s))) return rc;
    Plan P;
    const int save = h->prec;
    h->prec = kFP64;
    rc = prepare(h, 1, s, 0, 0, &P);
    h->prec = save;
    if (rc) return rc;
    launch_sketch_partials(P, v, nullptr, nullptr, P.cpart);
    launch_sketch_reduce(P, P.cpart, c, nullptr);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

int sfgmres_sketch_pattern(sfgmres_t h, int32_t s, int32_t* rows, int8_t* signs) {
    if (!h) return SFGMRES_ERR_INVALID_ARG;
    if (!rows || !signs) return fail(h, SFGMRES_ERR_INVALID_ARG, "NULL pointer");
    int rc = check_params(h, 1, s, 0);
    if (rc) return rc;
    CK(cudaSetDevice(h->dev));
    const int zeta = (h->kind == 1) ? 1 : h->zeta;
    int8_t* neg = nullptr;
    CK(cudaMalloc(&neg, (size_t)h->n * zeta));
    Plan dummy;
    launch_sketch_pattern(dummy, h->n, s, zeta, h->kind, h->seed, rows, neg, h->st);
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
    Plan P;
    P.n = h->n;
    P.rp = h->rp;
    P.col = h->col;
    P.val = h->val;
    P.vec = h->vec;
    P.Bn = h->Bn;
    P.nblk = h->nblk;
    P.st = h->st;
    launch_spmv_f64(P, xv, yv);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return SFGMRES_OK;
}

}  // extern "C"
