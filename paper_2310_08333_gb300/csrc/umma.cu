// Tensor-core sketch products of the Nystrom approximation (§2.2, sketch target of §3.3):
//   W = A Omega (m x s)   and   Y = A^T (D W) (n x s)
// as BF16 x BF16 -> FP32 GEMMs on the 5th-generation tensor cores (tcgen05.mma, accumulator in
// tensor memory), with operand tiles moved by 1-D bulk async copies.
//
// Precision.  A and Omega enter rounded to bfloat16 (the sketch only builds the preconditioner,
// so it approximates the Hessian of the bf16-rounded A; Omega's rounded values are written back
// so that the Nystrom core uses exactly the test matrix that was multiplied).  The intermediate
// D W is split into bfloat16 hi + lo parts that are stacked as one operand of 2 Np rows, so
// Y = A^T (D W) keeps about 2^-17 relative accuracy; FP32 accumulation throughout.
//
// Operand layout ("blocked"): an operand X (rows x K, K contiguous) is stored as tiles of RT rows
// x 64 k, each tile one contiguous block moved by one cp.async.bulk.  RT = 128 for the M-side
// operand (one tile per CTA row block) and RT = all N rows for the N-side operand.  Inside a
// tile, the 8-row x 16-byte core matrices follow each other along k first: core (g, c) (rows
// 8g..8g+7, k 8c..8c+7) starts at byte (8g + c) * 128, row r of it at r * 16, element k at
// (k mod 8) * 2.  This is the canonical non-swizzled K-major layout with 128 bytes between
// k-adjacent core matrices (leading byte offset) and 1024 bytes between row-adjacent groups
// (stride byte offset); one MMA of K = 16 spans two core-matrix columns, i.e. 256 bytes.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace genios {

constexpr int UM_THREADS = 192;       // warp 0 producer, warp 1 MMA issuer + TMEM owner, 2-5 epilogue
constexpr int UM_MAX_STAGES = 8;
constexpr uint32_t UM_TILE_A = 128 * 128;   // 128 rows x 64 bf16


// ------------------------------------------------------------------------------------------
// tcgen05 PTX
// ------------------------------------------------------------------------------------------
GENIOS_DEV uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family; base offset 0, no swizzle
    return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
GENIOS_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
GENIOS_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
GENIOS_DEV void tc_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
GENIOS_DEV void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
GENIOS_DEV void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
GENIOS_DEV void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
GENIOS_DEV void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------------------------------
// GEMM: out[split][row][col] = sum over this split's k tiles of Ablk[row, k] * Bblk[col, k]
// One CTA per (128-row tile, K split); rows of the output cover the padded M extent.
// ------------------------------------------------------------------------------------------
struct UmmaArgs {
    const unsigned char* A;   // blocked, RT = 128, mtiles x ktiles tiles of 16 KB
    const unsigned char* B;   // blocked, RT = N, ktiles tiles of N * 128 bytes
    float* out;               // [splits][mtiles * 128][N]
    int64_t mtiles, ktiles;
    int N, splits, stages;
    uint32_t tmem_cols;
    long long wait_limit;
    int* err;
};

__global__ void __launch_bounds__(UM_THREADS, 1) umma_gemm_kernel(UmmaArgs a) {
    extern __shared__ __align__(1024) unsigned char usm[];
    __shared__ __align__(8) uint64_t full[UM_MAX_STAGES];
    __shared__ __align__(8) uint64_t empty[UM_MAX_STAGES];
    __shared__ __align__(8) uint64_t accum;
    __shared__ uint32_t tmem_base;
    __shared__ int issued;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile = blockIdx.x % a.mtiles;
    const int split = (int)(blockIdx.x / a.mtiles);
    const int64_t kt0 = split * a.ktiles / a.splits, kt1 = (split + 1) * a.ktiles / a.splits;
    const int nk = (int)(kt1 - kt0);
    const uint32_t bytes_b = (uint32_t)a.N * 128u;
    const uint32_t stage_bytes = UM_TILE_A + bytes_b;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(usm) + 1023) & ~static_cast<uintptr_t>(1023));

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accum, 1);
        issued = 0;
        fence_mbar_init();
    }
    if (warp == 1) tc_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {   // producer: one A tile + the matching B tile per stage
            const uint64_t pol = l2_evict_first_policy();   // A tiles are read once per product
            int f = 0;
            for (; f < nk; ++f) {
                const int s = f % a.stages, use = f / a.stages;
                if (!mbar_wait_bounded(&empty[s], (uint32_t)((use & 1) ^ 1), a.wait_limit)) {
                    set_err(a.err, DERR_TIMEOUT_EMPTY);
                    break;
                }
                unsigned char* dst = smem + (size_t)s * stage_bytes;
                const int64_t kt = kt0 + f;
                mbar_arrive_expect_tx(&full[s], stage_bytes);
                bulk_g2s_hint(dst, a.A + (size_t)(tile * a.ktiles + kt) * UM_TILE_A, UM_TILE_A, &full[s], pol);
                bulk_g2s(dst + UM_TILE_A, a.B + (size_t)kt * bytes_b, bytes_b, &full[s]);
            }
            issued = f;
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = umma_idesc_bf16(128, a.N);
            int c = 0;
            for (; c < nk; ++c) {
                const int s = c % a.stages, use = c / a.stages;
                if (!mbar_wait_bounded(&full[s], (uint32_t)(use & 1), a.wait_limit)) {
                    set_err(a.err, DERR_TIMEOUT_FULL);
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
                const uint32_t sb = sa + UM_TILE_A;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t ad = umma_desc(sa + ks * 256, 128, 1024);
                    const uint64_t bd = umma_desc(sb + ks * 256, 128, 1024);
                    tc_mma(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                }
                tc_commit(&empty[s]);   // frees the stage when these MMAs have read it
            }
            tc_commit(&accum);          // all MMAs of this CTA
            // every MMA issued has written TMEM before it is released (drain limit: see common.cuh)
            if (!mbar_wait_bounded(&accum, 0, drain_limit(a.wait_limit))) set_err(a.err, DERR_TIMEOUT_FULL);
            // the last release of every stage has landed before the CTA can exit
            for (int s = 0; s < a.stages && s < c; ++s) {
                const int last = s + ((c - 1 - s) / a.stages) * a.stages;
                if (!mbar_wait_bounded(&empty[s], (uint32_t)((last / a.stages) & 1), drain_limit(a.wait_limit)))
                    set_err(a.err, DERR_TIMEOUT_EMPTY);
            }
        }
    } else {   // epilogue: TMEM lanes 32 (warp % 4) .. + 31 are rows of the tile
        const int q = warp & 3;
        bool ok = mbar_wait_bounded(&accum, 0, a.wait_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) set_err(a.err, DERR_TIMEOUT_FULL);
        } else {
            tc_fence_after();
            const int64_t row = tile * 128 + q * 32 + lane;
            float* o = a.out + ((int64_t)split * a.mtiles * 128 + row) * a.N;
            for (int c0 = 0; c0 < a.N; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                float4* o4 = reinterpret_cast<float4*>(o + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc(tmem, a.tmem_cols);
    }
    if (threadIdx.x == 0) {   // every bulk copy this CTA issued has landed before it exits
        const int f = issued;
        for (int s = 0; s < a.stages && s < f; ++s) {
            const int last = s + ((f - 1 - s) / a.stages) * a.stages;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((last / a.stages) & 1), drain_limit(a.wait_limit)))
                set_err(a.err, DERR_TIMEOUT_FULL);
        }
    }
}

// ------------------------------------------------------------------------------------------
// packing and finishing kernels
// ------------------------------------------------------------------------------------------
template <typename TA>
GENIOS_DEV float load_src(const TA* A, int64_t idx, const float* rs, int64_t row);
template <> GENIOS_DEV float load_src<float>(const float* A, int64_t idx, const float*, int64_t) { return A[idx]; }
template <> GENIOS_DEV float load_src<__nv_bfloat16>(const __nv_bfloat16* A, int64_t idx, const float*, int64_t) {
    return __bfloat162float(A[idx]);
}
template <> GENIOS_DEV float load_src<uint8_t>(const uint8_t* A, int64_t idx, const float* rs, int64_t row) {
    __nv_fp8_e4m3 q;
    q.__x = A[idx];
    return (float)q * rs[row];
}

// lo != 0: the remainder x - bf16(x), whose own bf16 rounding is the low half of a hi + lo split
GENIOS_DEV float lo_part(float x, int lo) {
    return lo ? x - __bfloat162float(__float2bfloat16_rn(x)) : x;
}

GENIOS_DEV uint4 pack8(const float (&v)[8]) {
    uint4 u;
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * i]);
        const __nv_bfloat16 hi = __float2bfloat16_rn(v[2 * i + 1]);
        w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
    u.x = w[0]; u.y = w[1]; u.z = w[2]; u.w = w[3];
    return u;
}

// A (m x n, row stride lda) -> blocked bf16 with rows = samples (M-side of W = A Omega).
template <typename TA>
__global__ void pack_rows_kernel(int64_t m, int64_t n, const TA* A, int64_t lda, const float* rs,
                                 int64_t rpad, int64_t kpad, unsigned char* out, int lo) {
    const int64_t kch = kpad / 8, total = rpad * kch;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / kch, k0 = (e % kch) * 8;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            v[t] = (row < m && k0 + t < n) ? lo_part(load_src<TA>(A, row * lda + k0 + t, rs, row), lo) : 0.0f;
        *reinterpret_cast<uint4*>(out + blk_off(row, k0, kpad / 64, 128)) = pack8(v);
    }
}

// A^T (n x m) -> blocked bf16 with rows = features (M-side of Y = A^T W'); consecutive threads
// take consecutive features so that the column reads of A coalesce.
template <typename TA>
__global__ void pack_cols_kernel(int64_t m, int64_t n, const TA* A, int64_t lda, const float* rs,
                                 int64_t rpad, int64_t kpad, unsigned char* out, int lo) {
    const int64_t total = rpad * (kpad / 8);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e % rpad, i0 = (e / rpad) * 8;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            v[t] = (j < n && i0 + t < m) ? lo_part(load_src<TA>(A, (i0 + t) * lda + j, rs, i0 + t), lo) : 0.0f;
        *reinterpret_cast<uint4*>(out + blk_off(j, i0, kpad / 64, 128)) = pack8(v);
    }
}

// Omega (n x s float, row-major) -> rounded in place to bfloat16 values and packed as the
// N-side operand (rows = the np >= s columns of Omega, k = feature).
__global__ void pack_omega_kernel(int64_t n, int sk, int np, float* Om, int64_t kpad, unsigned char* out) {
    const int64_t total = (int64_t)np * (kpad / 8);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % np);
        const int64_t j0 = (e / np) * 8;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float x = 0.0f;
            if (c < sk && j0 + t < n) {
                x = __bfloat162float(__float2bfloat16_rn(Om[(j0 + t) * sk + c]));
                Om[(j0 + t) * sk + c] = x;
            }
            v[t] = x;
        }
        *reinterpret_cast<uint4*>(out + blk_off(c, j0, kpad / 64, np)) = pack8(v);
    }
}

// W' = D (sum over splits of W) split into bf16 hi (rows 0..np-1) + lo (rows np..2np-1) of the
// N-side operand of the second product (k = sample).
__global__ void finish_w_kernel(int64_t m, int sk, int np, const float* part, int splits, int64_t mrows,
                                const float* d, int64_t kpad, unsigned char* out) {
    const int64_t total = (int64_t)np * (kpad / 8);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % np);
        const int64_t i0 = (e / np) * 8;
        float hi[8], lo[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int64_t i = i0 + t;
            float w = 0.0f;
            if (c < sk && i < m) {
                for (int z = 0; z < splits; ++z) w += part[((int64_t)z * mrows + i) * np + c];
                if (d) w *= d[i];
            }
            const float h = __bfloat162float(__float2bfloat16_rn(w));
            hi[t] = h;
            lo[t] = w - h;
        }
        *reinterpret_cast<uint4*>(out + blk_off(c, i0, kpad / 64, 2 * np)) = pack8(hi);
        *reinterpret_cast<uint4*>(out + blk_off(np + c, i0, kpad / 64, 2 * np)) = pack8(lo);
    }
}

// Y[j][c] = sum over splits of (hi + lo columns of the second product).
__global__ void finish_y_kernel(int64_t n, int sk, int np, const float* part, int splits, int64_t mrows,
                                float* Y) {
    const int64_t total = n * sk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / sk;
        const int c = (int)(e % sk);
        float y = 0.0f;
        for (int z = 0; z < splits; ++z) {
            const float* r = part + ((int64_t)z * mrows + j) * (2 * np);
            y += r[c] + r[np + c];
        }
        Y[e] = y;
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
static int64_t rup(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

static int sm_count_impl() {
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
    }
    return v;
}

int tc_sm_count() { return sm_count_impl(); }
static int sm_count() { return sm_count_impl(); }

static int stages_for(int N) {
    // two CTAs per SM: about 110 KB of operand stages each
    const int64_t sb = UM_TILE_A + (int64_t)N * 128;
    return (int)std::max<int64_t>(2, std::min<int64_t>(UM_MAX_STAGES, (110 * 1024) / sb));
}

int tc_splits_for(int64_t mtiles, int64_t ktiles) {
    const int64_t slots = 2 * (int64_t)sm_count();
    return (int)std::max<int64_t>(1, std::min<int64_t>(ktiles, slots / std::max<int64_t>(1, mtiles)));
}

TcPlan tc_plan(int64_t m, int64_t n, int sk) {
    TcPlan p{};
    p.m = m;
    p.n = n;
    p.sk = sk;
    p.np = (int)rup(sk, 16);
    p.rpad_m = rup(m, 128);
    p.kpad_n = rup(n, 64);
    p.rpad_n = rup(n, 128);
    p.kpad_m = rup(m, 64);
    p.splits1 = tc_splits_for(p.rpad_m / 128, p.kpad_n / 64);
    p.splits2 = tc_splits_for(p.rpad_n / 128, p.kpad_m / 64);
    p.ok = sk >= 1 && p.np <= 128;
    return p;
}

size_t tc_bytes(const TcPlan& p, size_t* off) {
    size_t o[6];
    size_t b = 0;
    auto take = [&](int i, size_t sz) { o[i] = b; b += (sz + 1023) & ~size_t(1023); };
    take(0, (size_t)p.rpad_m * p.kpad_n * 2);                  // A rows
    take(1, (size_t)p.rpad_n * p.kpad_m * 2);                  // A^T rows
    take(2, (size_t)p.np * p.kpad_n * 2);                      // Omega
    take(3, (size_t)2 * p.np * p.kpad_m * 2);                  // W' hi / lo
    take(4, std::max((size_t)p.splits1 * p.rpad_m * p.np, (size_t)p.splits2 * p.rpad_n * 2 * p.np) * 4);
    take(5, 256);                                              // error flag
    if (off)
        for (int i = 0; i < 6; ++i) off[i] = o[i];
    return b;
}

TcWork tc_carve(void* base, const TcPlan& p) {
    size_t off[6];
    tc_bytes(p, off);
    unsigned char* b = static_cast<unsigned char*>(base);
    TcWork w{};
    w.A_rows = b + off[0];
    w.A_cols = b + off[1];
    w.Om = b + off[2];
    w.W = b + off[3];
    w.part = reinterpret_cast<float*>(b + off[4]);
    w.err = reinterpret_cast<int*>(b + off[5]);
    return w;
}

cudaError_t tc_pack_a(const TcPlan& p, TcWork w, int src_prec, const void* A, int64_t lda,
                      const float* row_scale, cudaStream_t s, int lo) {
    const int T = 256;
    const int G = 4 * sm_count();
    if (src_prec == P_FP32) {
        pack_rows_kernel<float><<<G, T, 0, s>>>(p.m, p.n, static_cast<const float*>(A), lda, nullptr, p.rpad_m, p.kpad_n, w.A_rows, lo);
        pack_cols_kernel<float><<<G, T, 0, s>>>(p.m, p.n, static_cast<const float*>(A), lda, nullptr, p.rpad_n, p.kpad_m, w.A_cols, lo);
    } else if (src_prec == P_BF16) {
        auto Ab = static_cast<const __nv_bfloat16*>(A);
        pack_rows_kernel<__nv_bfloat16><<<G, T, 0, s>>>(p.m, p.n, Ab, lda, nullptr, p.rpad_m, p.kpad_n, w.A_rows, lo);
        pack_cols_kernel<__nv_bfloat16><<<G, T, 0, s>>>(p.m, p.n, Ab, lda, nullptr, p.rpad_n, p.kpad_m, w.A_cols, lo);
    } else if (src_prec == P_FP8) {
        auto Aq = static_cast<const uint8_t*>(A);
        pack_rows_kernel<uint8_t><<<G, T, 0, s>>>(p.m, p.n, Aq, lda, row_scale, p.rpad_m, p.kpad_n, w.A_rows, lo);
        pack_cols_kernel<uint8_t><<<G, T, 0, s>>>(p.m, p.n, Aq, lda, row_scale, p.rpad_n, p.kpad_m, w.A_cols, lo);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t tc_pack_omega(const TcPlan& p, TcWork w, float* Om, cudaStream_t s) {
    pack_omega_kernel<<<2 * sm_count(), 256, 0, s>>>(p.n, p.sk, p.np, Om, p.kpad_n, w.Om);
    return cudaGetLastError();
}

cudaError_t tc_gemm(const unsigned char* A, const unsigned char* B, float* out, int64_t mtiles,
                    int64_t ktiles, int N, int splits, int* err, long long wait_limit, cudaStream_t s) {
    UmmaArgs a{};
    a.A = A;
    a.B = B;
    a.out = out;
    a.mtiles = mtiles;
    a.ktiles = ktiles;
    a.N = N;
    a.splits = splits;
    a.stages = stages_for(N);
    a.tmem_cols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
    a.wait_limit = wait_limit;
    a.err = err;
    if (N < 16 || N > 256 || (N % 16) != 0 || splits < 1 || splits > ktiles) return cudaErrorInvalidValue;
    const size_t smem = (size_t)a.stages * (UM_TILE_A + (size_t)N * 128) + 1024;
    cudaError_t e = smem_optin<umma_gemm_kernel>();
    if (e != cudaSuccess) return e;
    umma_gemm_kernel<<<(unsigned)(mtiles * splits), UM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t tc_sketch(const TcPlan& p, TcWork w, const float* d, float* Y, long long wait_limit, cudaStream_t s) {
    if (!p.ok) return cudaErrorInvalidValue;
    cudaError_t e = tc_gemm(w.A_rows, w.Om, w.part, p.rpad_m / 128, p.kpad_n / 64, p.np, p.splits1, w.err,
                            wait_limit, s);
    if (e != cudaSuccess) return e;
    finish_w_kernel<<<2 * sm_count(), 256, 0, s>>>(p.m, p.sk, p.np, w.part, p.splits1, p.rpad_m, d, p.kpad_m, w.W);
    e = tc_gemm(w.A_cols, w.W, w.part, p.rpad_n / 128, p.kpad_m / 64, 2 * p.np, p.splits2, w.err, wait_limit, s);
    if (e != cudaSuccess) return e;
    finish_y_kernel<<<2 * sm_count(), 256, 0, s>>>(p.n, p.sk, p.np, w.part, p.splits2, p.rpad_n, Y);
    return cudaGetLastError();
}

cudaError_t batch_pack_lo(const TcPlan& p, TcWork w, const float* A, int64_t lda, cudaStream_t s) {
    return tc_pack_a(p, w, P_FP32, A, lda, nullptr, s, 1);
}

}  // namespace genios
