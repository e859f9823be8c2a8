// c = S v without any device allocation, for callers that cannot call cudaMalloc.
//
// Some callers of this library may not allocate device memory at the point where they need a sketch: code running
// inside a region whose memory plan is fixed in advance (a captured or replayed sequence of work, a real-time loop
// with a no-allocation rule), or a host application whose device memory is owned by another allocator or memory
// pool that must not be bypassed.  A solver handle allocates (CSR copy, gather lists, workspaces), so this entry
// point needs none: the per-block partial sums live in one file-scope static __device__ array of fixed size, which
// every GPU that loads the library holds until the process exits.  The caller passes only its input and output.
//
// The embedding is the same one a handle created with the same seed applies (same SplitMix64 draw rule, see
// sketch_column), so results agree with sfgmres_sketch_apply up to summation rounding.  Each CTA owns a block of
// columns, draws their rows on the fly, and sums its terms exactly in 64-bit fixed point relative to the block's
// largest exponent with shared-memory integer atomics (integer addition is order independent, so the result is
// deterministic); the block partials are then summed in block order.
#include "../../include/sfgmres.h"
#include "common.cuh"

#include <cmath>
#include <mutex>
#include <string>

namespace sfg {

// Largest number of (block, sketch row) partials the static scratch holds: 2^20 doubles = 8 MiB.
constexpr int64_t kNoallocScratch = int64_t(1) << 20;
constexpr int kNoallocMinCols = 1024;     // columns per block, at least
constexpr int kNoallocMaxCols = 65536;    // columns per block, at most (keeps the fixed-point headroom small)

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratch];

void set_global_error(const std::string& msg);  // api.cu: the message sfgmres_last_error(NULL) returns

__global__ void __launch_bounds__(512)
    k_noalloc_partials(int64_t n, int Bn, int s, int zeta, uint64_t seed, const double* __restrict__ v,
                       double* __restrict__ part) {
    extern __shared__ unsigned char smem_raw[];
    long long* acc = reinterpret_cast<long long*>(smem_raw);  // [s]
    int* cnt = reinterpret_cast<int*>(acc + s);               // [s]
    __shared__ int wmax[32], wcnt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * Bn;
    const int64_t c1 = min(n, c0 + Bn);
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        acc[r] = 0;
        cnt[r] = 0;
    }
    __syncthreads();
    // pass 1: terms per sketch row (for the overflow headroom) and the block's largest exponent
    int emax = 1;
    int rows[kMaxZeta], neg[kMaxZeta];
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        sketch_column(seed, j, zeta, s, rows, neg);
        for (int l = 0; l < zeta; ++l) atomicAdd(cnt + rows[l], 1);
        emax = max(emax, exp_of(v[j]));
    }
    __syncthreads();
    int cmax = 0;
    for (int r = threadIdx.x; r < s; r += blockDim.x) cmax = max(cmax, cnt[r]);
    emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
    cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cmax);
    if (lane == 0) {
        wmax[warp] = emax;
        wcnt[warp] = cmax;
    }
    __syncthreads();
    int Eb = 1, L = 0;
    for (int q = 0; q < nw; ++q) {
        Eb = max(Eb, wmax[q]);
        L = max(L, wcnt[q]);
    }
    int H = 0;
    while ((L >> H) >= 1023) ++H;  // |term| <= 2^53, so at most 1023 * 2^H terms keep every sum below 2^63
    // pass 2: exact fixed-point sums
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        const long long q = to_fixed(v[j], Eb, H);
        sketch_column(seed, j, zeta, s, rows, neg);
        for (int l = 0; l < zeta; ++l)
            atomicAdd(reinterpret_cast<unsigned long long*>(acc + rows[l]),
                      (unsigned long long)(neg[l] ? -q : q));
    }
    __syncthreads();
    const double unit = ldexp(1.0, Eb + H - 1075);
    for (int r = threadIdx.x; r < s; r += blockDim.x)
        part[(int64_t)blockIdx.x * s + r] = (Eb >= 2047) ? (double)NAN : (double)acc[r] * unit;
}

__global__ void k_noalloc_reduce(int nblk, int s, double scale, const double* __restrict__ part,
                                 double* __restrict__ c) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= s) return;
    double a = 0.0;
    for (int b = 0; b < nblk; ++b) a += part[(int64_t)b * s + r];
    c[r] = scale * a;
}

// Dynamic shared memory of k_noalloc_partials for s sketch rows: one 64-bit accumulator and one counter per row.
static size_t partials_smem(int s) { return (size_t)s * (sizeof(long long) + sizeof(int)); }

// Once per device, with that device current: look up the device address of the scratch array (cudaGetSymbolAddress;
// in host code the array's name is only a host-side stand-in) and allow k_noalloc_partials the dynamic shared memory
// of the largest sketch (4096 rows need 48 KiB, which with the kernel's static shared memory is above the default
// limit).  Both results are cached per device.
static cudaError_t device_setup(double** out) {
    static std::mutex mu;
    static double* cache[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) {
        e = cudaFuncSetAttribute((const void*)k_noalloc_partials, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)partials_smem(kMaxS));
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        cache[dev] = static_cast<double*>(p);
    }
    *out = cache[dev];
    return cudaSuccess;
}

// Launch with the error of this launch alone as the result (the launch API returns it; an error left behind by
// unrelated earlier work is neither reported nor cleared here).  A failed launch's own error is cleared.
template <typename... KArgs, typename... Args>
static cudaError_t launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                          Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

}  // namespace sfg

extern "C" int sfgmres_sketch_apply_noalloc(int64_t n, int32_t s, int32_t zeta, uint64_t sketch_seed,
                                            const double* v, double* c, void* stream) {
    using namespace sfg;
    if (!v || !c) {
        set_global_error("sfgmres_sketch_apply_noalloc: v and c must not be NULL");
        return SFGMRES_ERR_INVALID_ARG;
    }
    if (n < 1 || n > INT32_MAX) {
        set_global_error("sfgmres_sketch_apply_noalloc: n must be in [1, 2^31-1]");
        return SFGMRES_ERR_INVALID_ARG;
    }
    if (zeta < 1 || zeta > kMaxZeta || s < zeta || s > kMaxS) {
        set_global_error("sfgmres_sketch_apply_noalloc: need 1 <= zeta <= 16 and zeta <= s <= 4096");
        return SFGMRES_ERR_INVALID_ARG;
    }
    const int64_t max_blocks = kNoallocScratch / s;
    const int64_t max_n = max_blocks * kNoallocMaxCols;
    if (n > max_n) {
        set_global_error("sfgmres_sketch_apply_noalloc: n exceeds the static scratch limit (n <= 65536 * floor(2^20"
                         " / s) = " + std::to_string(max_n) + " for s = " + std::to_string(s) + ")");
        return SFGMRES_ERR_INVALID_ARG;
    }
    double* part = nullptr;
    cudaError_t e = device_setup(&part);
    if (e != cudaSuccess) {
        set_global_error(std::string("sfgmres_sketch_apply_noalloc: device set-up (cudaFuncSetAttribute / "
                                     "cudaGetSymbolAddress): ") + cudaGetErrorString(e));
        return SFGMRES_ERR_CUDA;
    }
    int64_t nblk = (n + kNoallocMinCols - 1) / kNoallocMinCols;
    if (nblk > max_blocks) nblk = max_blocks;
    int64_t Bn = (n + nblk - 1) / nblk;
    Bn = ((Bn + 31) / 32) * 32;
    nblk = (n + Bn - 1) / Bn;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = launch(k_noalloc_partials, (unsigned)nblk, 512, partials_smem(s), st, n, (int)Bn, (int)s, (int)zeta,
               sketch_seed, v, part);
    if (e != cudaSuccess) {
        set_global_error(std::string("sfgmres_sketch_apply_noalloc: launch of the block partials kernel: ") +
                         cudaGetErrorString(e));
        return SFGMRES_ERR_CUDA;
    }
    e = launch(k_noalloc_reduce, (unsigned)((s + 127) / 128), 128, 0, st, (int)nblk, (int)s,
               1.0 / std::sqrt((double)zeta), (const double*)part, c);
    if (e != cudaSuccess) {
        set_global_error(std::string("sfgmres_sketch_apply_noalloc: launch of the reduction kernel: ") +
                         cudaGetErrorString(e));
        return SFGMRES_ERR_CUDA;
    }
    return SFGMRES_OK;
}
