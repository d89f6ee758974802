// Common device helpers of the GeNIOS engine (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#define GENIOS_DEV __device__ __forceinline__

namespace genios {

// ------------------------------------------------------------------------------------------
// Precision tags
// ------------------------------------------------------------------------------------------
enum Prec { P_FP64 = 0, P_FP32 = 1, P_BF16 = 2, P_FP8 = 3, P_HILO = 4 };

// Storage element of A per precision and the number of elements in one 16-byte chunk.
template <int P> struct AStore;
template <> struct AStore<P_FP64> { using T = double;         static constexpr int VEC = 2;  };
template <> struct AStore<P_FP32> { using T = float;          static constexpr int VEC = 4;  };
template <> struct AStore<P_BF16> { using T = __nv_bfloat16;  static constexpr int VEC = 8;  };
template <> struct AStore<P_FP8>  { using T = uint8_t;        static constexpr int VEC = 16; };
template <> struct AStore<P_HILO> { using T = __nv_bfloat16;  static constexpr int VEC = 8;  };

// Value (vector) type per precision.
template <int P> struct VType { using T = float; };
template <> struct VType<P_FP64> { using T = double; };

inline int64_t elem_bytes(int P) {
    return P == P_FP64 ? 8 : P == P_FP32 ? 4 : P == P_FP8 ? 1 : 2;
}
// Leading dimension: rows start on 64-byte boundaries (16-byte chunks, whole sectors).
inline int64_t padded_lda(int P, int64_t n) {
    int64_t per = 64 / elem_bytes(P);
    return ((n + per - 1) / per) * per;
}

// ------------------------------------------------------------------------------------------
// Loss functors (§3.3): value, first and second derivative.
// ------------------------------------------------------------------------------------------
enum LossKind { LOSS_SQUARED = 0, LOSS_LOGISTIC = 1, LOSS_HUBER = 2 };

template <typename T> GENIOS_DEV T sigmoid_(T w);
template <> GENIOS_DEV float sigmoid_<float>(float w) { return 1.0f / (1.0f + expf(-w)); }
template <> GENIOS_DEV double sigmoid_<double>(double w) { return 1.0 / (1.0 + exp(-w)); }

template <typename T>
GENIOS_DEV void loss_eval(int loss, T t, T& l0, T& l1, T& l2) {
    if (loss == LOSS_SQUARED) {
        l0 = T(0.5) * t * t;
        l1 = t;
        l2 = T(1);
    } else if (loss == LOSS_HUBER) {   // §4.4: t^2 inside |t| <= 1, 2|t| - 1 beyond
        const T at = t < T(0) ? -t : t;
        if (at <= T(1)) {
            l0 = t * t;
            l1 = T(2) * t;
            l2 = T(2);
        } else {
            l0 = T(2) * at - T(1);
            l1 = t < T(0) ? T(-2) : T(2);
            l2 = T(0);
        }
    } else {
        T s = sigmoid_<T>(t);
        // log(1 + e^t) = max(t, 0) + log1p(e^{-|t|})
        T at = t < T(0) ? -t : t;
        l0 = (t > T(0) ? t : T(0)) + log1p(exp(-at));
        l1 = s;
        l2 = s * (T(1) - s);
    }
}

// l'(t) alone, the same value loss_eval gives as l1
template <typename T>
GENIOS_DEV T loss_d1(int loss, T t) {
    if (loss == LOSS_SQUARED) return t;
    if (loss == LOSS_HUBER) {
        const T at = t < T(0) ? -t : t;
        return at <= T(1) ? T(2) * t : (t < T(0) ? T(-2) : T(2));
    }
    return sigmoid_<T>(t);
}

// Fenchel conjugate of the loss (App. A), +inf outside the domain.
GENIOS_DEV double loss_conj(int loss, double v) {
    if (loss == LOSS_SQUARED) return 0.5 * v * v;
    if (loss == LOSS_HUBER) return fabs(v) <= 2.0 ? 0.25 * v * v : __longlong_as_double(0x7ff0000000000000LL);
    if (v < 0.0 || v > 1.0) return __longlong_as_double(0x7ff0000000000000LL);
    double a = v > 0.0 ? v * log(v) : 0.0;
    double b = v < 1.0 ? (1.0 - v) * log1p(-v) : 0.0;
    return a + b;
}

// ------------------------------------------------------------------------------------------
// 16-byte chunk decoding into float / double lanes
// ------------------------------------------------------------------------------------------
GENIOS_DEV void decode_chunk(const uint4& c, float (&f)[4]) {
    f[0] = __uint_as_float(c.x); f[1] = __uint_as_float(c.y);
    f[2] = __uint_as_float(c.z); f[3] = __uint_as_float(c.w);
}
GENIOS_DEV void decode_chunk(const uint4& c, double (&f)[2]) {
    f[0] = __hiloint2double(c.y, c.x);
    f[1] = __hiloint2double(c.w, c.z);
}
GENIOS_DEV float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
GENIOS_DEV float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
GENIOS_DEV void decode_chunk(const uint4& c, float (&f)[8]) {
    f[0] = bf16lo(c.x); f[1] = bf16hi(c.x); f[2] = bf16lo(c.y); f[3] = bf16hi(c.y);
    f[4] = bf16lo(c.z); f[5] = bf16hi(c.z); f[6] = bf16lo(c.w); f[7] = bf16hi(c.w);
}
GENIOS_DEV void fp8x4_to_float(uint32_t w, float* f) {
    __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&h0));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&h1));
    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
}
GENIOS_DEV void decode_chunk(const uint4& c, float (&f)[16]) {
    fp8x4_to_float(c.x, f + 0); fp8x4_to_float(c.y, f + 4);
    fp8x4_to_float(c.z, f + 8); fp8x4_to_float(c.w, f + 12);
}

// Packed float32 pairs (sm_100 family): two IEEE float32 FMAs / adds per instruction on a
// 64-bit register pair.  Packing adjacent values lets the compiler keep them in a register pair.
GENIOS_DEV uint64_t f2pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
GENIOS_DEV float2 f2unpack(uint64_t r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
GENIOS_DEV uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
GENIOS_DEV uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ------------------------------------------------------------------------------------------
// PTX: shared-memory addresses, mbarriers, bulk async copies (sm_90+)
// ------------------------------------------------------------------------------------------
GENIOS_DEV uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
GENIOS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
GENIOS_DEV void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
GENIOS_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
GENIOS_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
GENIOS_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Floor of the limit on the waits with which a CTA drains its own asynchronous work before it
// releases the memory that work writes: bulk copies landing in its shared memory, MMAs writing
// its tensor memory.  About one second at the SM clock.  A caller's short device wait limit ends
// the waits on other threads and CTAs early, never these: that work always completes (each copy
// and MMA was issued against memory the CTA still holds), and only its completion makes the
// release safe.
constexpr long long DRAIN_MIN_CYCLES = 1LL << 31;
GENIOS_DEV long long drain_limit(long long limit) { return limit > DRAIN_MIN_CYCLES ? limit : DRAIN_MIN_CYCLES; }

// Bounded wait: returns false when `limit` clock cycles pass without completion.
GENIOS_DEV bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
// 1-D bulk copy global -> shared with transaction-count completion on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
GENIOS_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// L2 policy for data read once per pass (the streamed matrix): its lines are evicted first, so a
// pass over a matrix much larger than L2 does not displace the small working set (vectors,
// partial sums, the preconditioner) that the kernels around it reuse.
GENIOS_DEV uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// bulk_g2s with an L2 cache-policy hint
GENIOS_DEV void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
GENIOS_DEV void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Named barrier over `nthreads` threads that also ORs a predicate across them.
GENIOS_DEV bool named_bar_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
GENIOS_DEV uint4 ld_shared_v4(const void* p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

// ------------------------------------------------------------------------------------------
// Reductions
// ------------------------------------------------------------------------------------------
template <typename T> GENIOS_DEV T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> GENIOS_DEV T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Sum NV doubles over the block; result valid in every thread.  blockDim.x multiple of 32,
// <= 1024.  The shared scratch (32 x NV doubles) is owned here, sized by the template.
template <int NV>
GENIOS_DEV void block_sum(double (&v)[NV]) {
    __shared__ double sh[32 * NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = lane < nw ? sh[k * 32 + lane] : 0.0;
        v[k] = warp_sum(t);
    }
    __syncthreads();
}

// Deterministic grid-wide sum of NV doubles: every block writes its block sum into
// part[blockIdx.x * NV + k]; the last block to finish sums the partials in block order and
// returns true (result in `out`, valid in all its threads).  The counter is reset for reuse.
template <int NV>
GENIOS_DEV bool grid_sum(double (&v)[NV], double* part, unsigned* counter, double (&out)[NV]) {
    block_sum<NV>(v);
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * NV + k] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    // fixed order: thread t sums blocks t, t + blockDim, ...; then a fixed-shape tree
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + (size_t)b * NV + k);
    }
    block_sum<NV>(acc);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = acc[k];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Same as grid_sum but the last block also gets a max over blocks of NM doubles.
template <int NV, int NM>
GENIOS_DEV bool grid_sum_max(double (&v)[NV], double (&mx)[NM], double* part, unsigned* counter,
                             double (&out)[NV], double (&outmx)[NM]) {
    constexpr int N = NV + NM;
    __shared__ double sh[32 * N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
#pragma unroll
    for (int k = 0; k < NM; ++k) mx[k] = warp_max(mx[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
#pragma unroll
        for (int k = 0; k < NM; ++k) sh[(NV + k) * 32 + wid] = mx[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nw ? sh[k * 32 + lane] : 0.0);
#pragma unroll
    for (int k = 0; k < NM; ++k) mx[k] = warp_max(lane < nw ? sh[(NV + k) * 32 + lane] : -1e300);
    __syncthreads();
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * N + k] = v[k];
#pragma unroll
        for (int k = 0; k < NM; ++k) part[(size_t)blockIdx.x * N + NV + k] = mx[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV], am[NM];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) am[k] = -1e300;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + (size_t)b * N + k);
#pragma unroll
        for (int k = 0; k < NM; ++k) am[k] = fmax(am[k], __ldcg(part + (size_t)b * N + NV + k));
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
#pragma unroll
    for (int k = 0; k < NM; ++k) am[k] = warp_max(am[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = acc[k];
#pragma unroll
        for (int k = 0; k < NM; ++k) sh[(NV + k) * 32 + wid] = am[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = warp_sum(lane < nw ? sh[k * 32 + lane] : 0.0);
#pragma unroll
    for (int k = 0; k < NM; ++k) outmx[k] = warp_max(lane < nw ? sh[(NV + k) * 32 + lane] : -1e300);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Bounds self-checks (diagnostic builds with -DGENIOS_CHECKED): an access that would fall
// outside its buffer is skipped and its (line, index, length) recorded in dbg[0..3]; normal
// builds compile the checks away.
#ifdef GENIOS_CHECKED
GENIOS_DEV bool gchk(long long* dbg, int line, long long idx, long long len) {
    if (idx >= 0 && idx < len) return true;
    if (dbg != nullptr && atomicCAS(reinterpret_cast<unsigned long long*>(dbg), 0ull,
                                    (unsigned long long)line) == 0ull) {
        dbg[1] = idx;
        dbg[2] = len;
        dbg[3] = (long long)blockIdx.x * 4096 + threadIdx.x;
    }
    return false;
}
#define GCHK(dbg, idx, len) ::genios::gchk((dbg), __LINE__, (long long)(idx), (long long)(len))
#else
#define GCHK(dbg, idx, len) true
#endif

// Error codes written by kernels into the context's device error word.
enum DevErr { DERR_NONE = 0, DERR_TIMEOUT_FULL = 1, DERR_TIMEOUT_EMPTY = 2, DERR_CHOL = 3,
              DERR_NUMERIC = 4 };

GENIOS_DEV void set_err(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace genios
