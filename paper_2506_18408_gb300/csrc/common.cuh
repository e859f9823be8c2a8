// Shared device helpers and solver-state layouts of the sketched-FGMRES CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace sfg {

constexpr int kWarp = 32;
constexpr int kMaxTrunc = 8;    // largest Arnoldi truncation depth t
constexpr int kMaxZeta = 16;    // largest number of nonzeros per sketch column
constexpr int kMaxS = 4096;     // largest sketch size
constexpr int kMaxM = 1024;     // largest inner basis size
constexpr int kBlockRowsMax = 8192;  // rows per row block (local sketch offsets need <= 15 bits)
constexpr int kQrCluster = 8;        // CTAs of the cluster that runs the sketched QR update

// ------------------------------------------------------------------------------------------------------------
// Precision traits.  VT: storage type of inner basis vectors; AT: arithmetic / accumulation type; MT: matrix values.
template <typename T> struct Num;
template <> struct Num<double> {
    __device__ __forceinline__ static double to_f(double x) { return x; }
};
template <> struct Num<float> {
    __device__ __forceinline__ static float to_f(float x) { return x; }
};

__device__ __forceinline__ double load_as(const double* p, double) { return __ldg(p); }
__device__ __forceinline__ float load_as(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float load_as(const __nv_bfloat16* p, float) { return __bfloat162float(*p); }
__device__ __forceinline__ double ld_plain(const double* p) { return *p; }
__device__ __forceinline__ float ld_plain(const float* p) { return *p; }
__device__ __forceinline__ float ld_plain(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Loads and stores with L2 eviction priority "last" (policy from l2_keep_policy): for vectors that a later phase or
// step reads again (the Arnoldi window rows, w', the next basis vector), so that the matrix stream, read once per
// step, is evicted before them.
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Eviction priority "first", for the last read of such a vector (it then leaves L2 before the ones still needed).
__device__ __forceinline__ unsigned long long l2_drop_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// ld_keep(p, pol) loads with the L2 policy pol (from l2_keep_policy or l2_drop_policy).
__device__ __forceinline__ double ld_keep(const double* p, unsigned long long pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_keep(const float* p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_keep(const __nv_bfloat16* p, unsigned long long pol) {
    unsigned short v;
    asm volatile("ld.global.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return __bfloat162float(__ushort_as_bfloat16(v));
}
__device__ __forceinline__ void st_keep(double* p, double v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float* p, float v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(__nv_bfloat16* p, float v, unsigned long long pol) {
    const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(b), "l"(pol) : "memory");
}

// Value as it will read back after store_as (identity except for BF16 rounding).
__device__ __forceinline__ double fma_as(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_as(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double stored_value(double v, const double*) { return v; }
__device__ __forceinline__ float stored_value(float v, const float*) { return v; }
__device__ __forceinline__ float stored_value(float v, const __nv_bfloat16*) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// x * 2^p for FP64 with integer operations only (no FP64 instruction): exact for normal results; zero, Inf and
// NaN pass through; a result below the normal range is flushed to a signed zero (such entries are below 2^-1022
// times the vector's norm and do not matter), one above it becomes a signed infinity.
__device__ __forceinline__ double mul_pow2(double x, int p) {
    const long long bits = __double_as_longlong(x);
    const long long sign = bits & (long long)0x8000000000000000ull;
    const int e = (int)((bits >> 52) & 0x7FF);
    const int ne = e + p;
    long long outb = bits + ((long long)p << 52);
    if (e == 0x7FF) outb = bits;
    else if (e == 0 || ne <= 0) outb = sign;
    else if (ne >= 0x7FF) outb = sign | 0x7FF0000000000000ll;
    return __longlong_as_double(outb);
}

__device__ __forceinline__ void store_as(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_as(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_as(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// ------------------------------------------------------------------------------------------------------------
// Deterministic reductions (fixed shuffle trees, fixed shared-memory order).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over all threads of the block; result valid in every thread.  `red` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T r = (lane < nw) ? red[lane] : T(0);
    r = warp_sum(r);
    return r;
}

// ------------------------------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014), counter form: output k of the stream started at state `seed`.
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_draw(uint64_t seed, uint64_t k) {
    return sm64_mix(seed + (k + 1ull) * 0x9E3779B97F4A7C15ull);
}

// Rows and signs of sketch column j (zeta distinct rows in [0, s)).  Draw rule: slot q = j*zeta + l takes its row
// from outputs 128q + 2a for attempts a = 0..63 (first row unused by the column's earlier slots; after 64
// collisions, the next free row cyclically after the last candidate), row = ((h >> 32) * s) >> 32, and its sign
// from bit 63 of output 128q + 1 (0 = +).
__device__ __forceinline__ void sketch_column(uint64_t seed, int64_t j, int zeta, int s, int* rows, int* neg) {
    for (int l = 0; l < zeta; ++l) {
        const uint64_t base = (uint64_t)(j * zeta + l) * 128ull;
        int cand = 0;
        bool dup = true;
        for (int a = 0; a < 64 && dup; ++a) {
            const uint64_t h = sm64_draw(seed, base + 2ull * (uint64_t)a);
            cand = (int)(((h >> 32) * (uint64_t)s) >> 32);
            dup = false;
            for (int q = 0; q < l; ++q) dup |= (rows[q] == cand);
        }
        while (dup) {
            cand = (cand + 1 == s) ? 0 : cand + 1;
            dup = false;
            for (int q = 0; q < l; ++q) dup |= (rows[q] == cand);
        }
        rows[l] = cand;
        neg[l] = (int)(sm64_draw(seed, base + 1ull) >> 63);
    }
}

// ------------------------------------------------------------------------------------------------------------
// 64-bit fixed-point image of w relative to the block exponent Eb (max biased exponent in the block, >= 1):
// w ~= q * 2^(Eb + H - 1075), |q| <= 2^53, rounded to nearest (ties away from zero).  Integer operations only.
__device__ __forceinline__ long long to_fixed(double w, int Eb, int H) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
    const int e = (int)((bits >> 52) & 0x7FFull);
    unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
    int ee = e;
    if (e != 0) M |= (1ull << 52);
    else ee = 1;
    const int d = Eb - ee + H;
    unsigned long long q;
    if (d <= 0) q = M;
    else if (d >= 55) q = 0;
    else q = (M + (1ull << (d - 1))) >> d;
    return (bits >> 63) ? -(long long)q : (long long)q;
}

// FP32 analogue: w ~= q * 2^(Eb + H - 179) with |q| <= 2^53 (the 24-bit significand placed 29 bits up, so values
// within 2^29 of the block maximum are represented exactly).
__device__ __forceinline__ long long to_fixed(float w, int Eb, int H) {
    const unsigned bits = __float_as_uint(w);
    const int e = (int)((bits >> 23) & 0xFFu);
    unsigned long long M = (unsigned long long)(bits & 0x7FFFFFu);
    int ee = e;
    if (e != 0) M |= (1ull << 23);
    else ee = 1;
    M <<= 29;
    const int d = Eb - ee + H;
    unsigned long long q;
    if (d <= 0) q = M;
    else if (d >= 55) q = 0;
    else q = (M + (1ull << (d - 1))) >> d;
    return (bits >> 31) ? -(long long)q : (long long)q;
}

__device__ __forceinline__ int exp_of(float w) {
    const int e = (int)((__float_as_uint(w) >> 23) & 0xFFu);
    return e > 0 ? e : 1;
}

// Value of one unit of the fixed-point image: 2^(Eb + H - 1075) for FP64 data, 2^(Eb + H - 179) for FP32 data.
__device__ __forceinline__ double fixed_unit(double, int Eb, int H) { return ldexp(1.0, Eb + H - 1075); }
__device__ __forceinline__ double fixed_unit(float, int Eb, int H) { return ldexp(1.0, Eb + H - 179); }
__device__ __forceinline__ bool exp_nonfinite(double, int Eb) { return Eb >= 2047; }
__device__ __forceinline__ bool exp_nonfinite(float, int Eb) { return Eb >= 255; }

__device__ __forceinline__ int exp_of(double w) {
    const int e = (int)(((unsigned long long)__double_as_longlong(w) >> 52) & 0x7FFull);
    return e > 0 ? e : 1;
}

// ------------------------------------------------------------------------------------------------------------
// Sketch gather lists.  For row block b and sketch row r the list holds one 16-bit entry per nonzero S_rj with j in
// the block: bits 0..14 the offset of j in the block, bit 15 the sign.  The lists of the 32 rows of group g = r / 32
// are interleaved in 16-byte units (unit u of lane r % 32 at unit index seg[b*ng + g] + 32u + r % 32, ng = ceil(s /
// 32)) and padded to the group's longest list with entries that point at the block's zero slot (offset Bn), so a
// warp reads them with contiguous 16-byte loads and no bounds checks.
template <typename T>
__device__ __forceinline__ T sum8(const uint4 d, const T* __restrict__ x) {
    const unsigned w[4] = {d.x, d.y, d.z, d.w};
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const unsigned en = (w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
        const T v = x[en & 0x7fffu];
        acc += (en & 0x8000u) ? -v : v;
    }
    return acc;
}

// Sum of +-x[offset] over the gather list of one lane of a group (E units of 8 entries, unit u at unit index
// u0 + 32u + lane: the group's lists interleaved, so a warp's loads are contiguous), in list order (deterministic),
// four 16-byte loads in flight.
template <typename T>
__device__ __forceinline__ T sum_group(const uint16_t* __restrict__ ent, int u0, int E, int lane,
                                       const T* __restrict__ x) {
    const uint4* p = reinterpret_cast<const uint4*>(ent) + u0 + lane;
    T acc = T(0);
    int u = 0;
    for (; u + 4 <= E; u += 4) {
        uint4 d[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = __ldg(p + 32 * (u + k));
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += sum8(d[k], x);
    }
    for (; u < E; ++u) acc += sum8(__ldg(p + 32 * u), x);
    return acc;
}

// ------------------------------------------------------------------------------------------------------------
// Device-resident solver state (one instance per handle).
struct CycleState {
    int stopped;   // the inner cycle has ended (written only by the sketched-QR kernel)
    int k;         // accepted inner basis size
    int reason;    // 1 C1, 2 C2, 3 C3, 4 Arnoldi breakdown, 5 degenerate, 6 non-finite value
    int c3_on;     // rule C3 active for this cycle
    int brk_step;  // first step i whose input basis vector u_i has zero (or non-finite) norm; INT_MAX if none
    int brk_reason;  // 4 zero norm, 6 non-finite
    int pad0, pad1;
    double dmax, dmin;    // extremes of |r_ll| for the condition proxy
    double rho;           // sketched residual of the last accepted column
    double c3_scale;      // FFOM residual of the previous outer step (beta at the first)
    double c3_tol;        // tol * ||b||
    double cond_thr;
};

struct OuterState {
    int j;            // index of the current outer step (0-based)
    int conv_est;     // the Givens estimate met the tolerance at the last step
    int breakdown;    // h_{j+1,j} == 0 (exact) at the last step
    int nan;          // NaN/Inf seen in a reduction
    int sync_fail;    // the fused inner step's grid-wide wait gave up during the last inner cycle
    double beta;      // ||r0||
    double bnorm;     // ||b||
    double est;       // |g_{j+1}|
    double ffom;      // |g_{j+1}| / |c_j| (FFOM residual, Eq. 4)
    double true_res2; // ||b - A x||^2 of the last recomputation
    double tol_abs;   // tol * ||b||
};

}  // namespace sfg
