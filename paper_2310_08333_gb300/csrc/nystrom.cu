// Randomized Nystrom approximation of A^T diag(d) A (§2.2, §3.3) and the test matrix (sm_103a).
//
//   Omega   : Philox4x32-10 (Salmon et al. 2011) + Box-Muller standard normals, made orthonormal
//             by CholeskyQR2 once per data set.
//   sketch  : W = A Omega (m x s), W <- diag(d) W, Y = A^T W (n x s): tensor-core GEMMs
//             (umma.cu) for float value types, the tiled CUDA-core GEMMs below for float64.
//   core    : eta = sqrt(n) eps ||Y||_F; Y_eta = Y + eta Omega; G = Omega^T Y_eta (FP64 sums);
//             G = C^T C (FP64 Cholesky, one CTA, eta x 10 and retry on failure);
//             B = Y_eta C^{-1}; B^T B = V Sigma^2 V^T by cyclic Jacobi with round-robin parallel
//             ordering (Golub & Van Loan §8.5) in the value type, one CTA, warm-started from
//             the previous sketch's V when the test matrix is reused; one Newton-Schulz step
//             re-orthogonalises V; in float32 the eigenvalues are refined by float64 Rayleigh
//             quotients; U = B V Sigma^{-1}; lam = max(Sigma^2 - eta, 0), sorted descending.
//   adaptive: the power steps that estimate ||A^T diag(d) A - U diag(lam) U^T|| for the
//             adaptive sketch size (nys_error_step, nys_scale).
// The shift uses the machine epsilon of the value type (float64 or float32).
#include "common.cuh"
#include "internal.h"

#include <cmath>
#include <cstdint>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace genios {

static bool sync_check();

// ------------------------------------------------------------------------------------------
// Philox4x32-10
// ------------------------------------------------------------------------------------------
GENIOS_DEV uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
    }
    return c;
}

__global__ void philox_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                              uint32_t k1, int64_t nb, uint32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 r = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), make_uint2(k0, k1));
        out[4 * i + 0] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

template <typename VT>
__global__ void omega_kernel(int64_t total, uint32_t sid, uint32_t k0, uint32_t k1, VT* Om) {
    const int64_t nb = (total + 3) / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 r = philox4x32_10(make_uint4((uint32_t)i, sid, 0u, 0u), make_uint2(k0, k1));
        const double two32 = 4294967296.0;
        const double ua = ((double)r.x + 0.5) / two32, ub = ((double)r.y + 0.5) / two32;
        const double uc = ((double)r.z + 0.5) / two32, ud = ((double)r.w + 0.5) / two32;
        const double ra = sqrt(-2.0 * log(ua)), rb = sqrt(-2.0 * log(uc));
        double sa, ca, sb, cb;
        sincospi(2.0 * ub, &sa, &ca);
        sincospi(2.0 * ud, &sb, &cb);
        const double g[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = 4 * i + q;
            if (e < total) Om[e] = (VT)g[q];
        }
    }
}

cudaError_t philox_blocks(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1, int64_t nblocks, uint32_t* out, cudaStream_t s) {
    int grid = (int)std::min<int64_t>(1024, (nblocks + 255) / 256);
    if (grid < 1) grid = 1;
    philox_kernel<<<grid, 256, 0, s>>>(c0, c1, c2, c3, k0, k1, nblocks, out);
    return cudaGetLastError();
}

cudaError_t omega_fill(bool dbl, int64_t n, int sk, uint64_t seed, uint32_t sid, void* Om,
                       cudaStream_t s) {
    const int64_t total = n * (int64_t)sk;
    int grid = (int)std::min<int64_t>(2048, ((total + 3) / 4 + 255) / 256);
    if (grid < 1) grid = 1;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    if (dbl) omega_kernel<double><<<grid, 256, 0, s>>>(total, sid, k0, k1, static_cast<double*>(Om));
    else omega_kernel<float><<<grid, 256, 0, s>>>(total, sid, k0, k1, static_cast<float*>(Om));
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Sketch GEMMs (CUDA cores): W = diag(d) A Omega and Y = A^T W.
// 64 x 64 output tiles, K tiles of 32, 256 threads, 4 x 4 outputs per thread.
// ------------------------------------------------------------------------------------------
template <int P> GENIOS_DEV float load_a(const void* A, int64_t idx);
template <> GENIOS_DEV float load_a<P_FP32>(const void* A, int64_t idx) { return static_cast<const float*>(A)[idx]; }
template <> GENIOS_DEV float load_a<P_BF16>(const void* A, int64_t idx) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(A)[idx]);
}
template <> GENIOS_DEV float load_a<P_FP8>(const void* A, int64_t idx) {
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<const uint8_t*>(A)[idx], __NV_E4M3);
    return __half2float(*reinterpret_cast<__half*>(&h));
}

template <int P, typename VT>
GENIOS_DEV VT load_av(const void* A, int64_t idx) {
    if constexpr (P == P_FP64) return static_cast<const double*>(A)[idx];
    else return (VT)load_a<P>(A, idx);
}

constexpr int GT = 64, GK = 32;

// W[i, c] = d_i * scale_i * sum_k A[i, k] Omega[k, c]
template <int P, typename VT>
__global__ void __launch_bounds__(256) sketch_a_omega(int64_t m, int64_t n, int sk, const void* A,
                                                     int64_t lda, const float* rs, const VT* d,
                                                     const VT* Om, VT* W) {
    __shared__ VT As[GK][GT + 1];  // [k][i]
    __shared__ VT Bs[GK][GT];      // [k][c]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t i0 = (int64_t)blockIdx.x * GT;
    const int c0 = blockIdx.y * GT;
    VT acc[4][4] = {};
    for (int64_t k0 = 0; k0 < n; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int ii = e / GK, kk = e % GK;
            const int64_t i = i0 + ii, k = k0 + kk;
            As[kk][ii] = (i < m && k < n) ? load_av<P, VT>(A, i * lda + k) : VT(0);
        }
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int kk = e / GT, cc = e % GT;
            const int64_t k = k0 + kk;
            const int c = c0 + cc;
            Bs[kk][cc] = (k < n && c < sk) ? Om[k * sk + c] : VT(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GK; ++kk) {
            VT a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty * 4 + r;
        if (i >= m) continue;
        VT sc = d != nullptr ? d[i] : VT(1);
        if constexpr (P == P_FP8) sc *= (VT)rs[i];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cc = c0 + tx * 4 + c;
            if (cc < sk) W[i * sk + cc] = acc[r][c] * sc;
        }
    }
}

// Y[j, c] = sum_i A[i, j] scale_i W[i, c]
template <int P, typename VT>
__global__ void __launch_bounds__(256) sketch_at_w(int64_t m, int64_t n, int sk, const void* A,
                                                  int64_t lda, const float* rs, const VT* W, VT* Y) {
    __shared__ VT As[GK][GT + 1];  // [i][j]
    __shared__ VT Bs[GK][GT];      // [i][c]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t j0 = (int64_t)blockIdx.x * GT;
    const int c0 = blockIdx.y * GT;
    VT acc[4][4] = {};
    for (int64_t i0 = 0; i0 < m; i0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int ii = e / GT, jj = e % GT;
            const int64_t i = i0 + ii, j = j0 + jj;
            VT v = (i < m && j < n) ? load_av<P, VT>(A, i * lda + j) : VT(0);
            if constexpr (P == P_FP8) v = (i < m) ? v * (VT)rs[i] : v;
            As[ii][jj] = v;
        }
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int ii = e / GT, cc = e % GT;
            const int64_t i = i0 + ii;
            const int c = c0 + cc;
            Bs[ii][cc] = (i < m && c < sk) ? W[i * sk + c] : VT(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < GK; ++ii) {
            VT a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[ii][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[ii][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t j = j0 + ty * 4 + r;
        if (j >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cc = c0 + tx * 4 + c;
            if (cc < sk) Y[j * sk + cc] = acc[r][c];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Tall-skinny helpers
// ------------------------------------------------------------------------------------------
// sum of squares of an n x s matrix -> out (double), deterministic two-level
template <typename VT>
__global__ void sumsq_kernel(int64_t total, const VT* X, double* part, unsigned* counter, double* out) {
    double v[1] = {0.0};
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)X[e];
        v[0] += x * x;
    }
    double o[1];
    if (grid_sum<1>(v, part, counter, o))
        if (threadIdx.x == 0) *out = o[0];
}

// The shifted sketch Y_eta = Y + eta Omega (§2.2) is never stored: the kernels that read it form
// it on the fly as fma(eta, Omega, Y), the same value type rounding wherever it is read.
// eta = c_eta sqrt(||Y||_F^2), c_eta = sqrt(n) eps mult (mult grows by 10x per failed attempt).

// 4-wide value-type vector (16 bytes for float, 32 for double)
template <typename VT> struct alignas(4 * sizeof(VT)) TsVec4 { VT v[4]; };

// Gram partials: part[b][a*s + c] = sum over block b's rows j of X[j,a] * Y'[j,c], with
// Y' = Y + eta Yadd when Yadd is given (block 0 then stores eta).  A block takes a contiguous
// share of the rows and stages them GR_ROWS at a time in shared memory (rows padded to a multiple
// of 4 entries); each thread owns up to GR_TILES 4 x 4 tiles of the s x s output (s <= 128) and
// accumulates them in the value type over the block's rows: per row, one 4-wide load of each
// operand per tile feeds 16 FMAs.  The partials are written as float64.
constexpr int GR_THREADS = 256, GR_ROWS = 32;
constexpr int GR_TILES = (32 * 32 + GR_THREADS - 1) / GR_THREADS;   // (s/4)^2 tiles, s <= 128
template <typename VT>
static size_t gram_smem(int sk) { return (size_t)2 * GR_ROWS * ((sk + 3) & ~3) * sizeof(VT); }
template <typename VT>
__global__ void __launch_bounds__(GR_THREADS) gram_partial(int64_t n, int sk, const VT* X, const VT* Y,
                                                          const VT* Yadd, const double* fro2, double c_eta,
                                                          double* eta_out, double* part) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int ldr = (sk + 3) & ~3;
    VT* xs = reinterpret_cast<VT*>(gsm);   // GR_ROWS x ldr
    VT* ys = xs + GR_ROWS * ldr;           // GR_ROWS x ldr
    const int ncg = ldr / 4;
    const int ntile = ncg * ncg;
    const VT eta = Yadd ? (VT)(c_eta * sqrt(*fro2)) : VT(0);
    if (Yadd && blockIdx.x == 0 && threadIdx.x == 0) *eta_out = (double)eta;
    const int64_t rows_per_block = (n + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t j1 = min(n, j0 + rows_per_block);
    VT acc[GR_TILES][4][4];
#pragma unroll
    for (int t = 0; t < GR_TILES; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[t][i][c] = VT(0);
    for (int64_t jt = j0; jt < j1; jt += GR_ROWS) {
        const int rows = (int)min((int64_t)GR_ROWS, j1 - jt);
        __syncthreads();   // the previous chunk's reads are done
        for (int e = threadIdx.x; e < GR_ROWS * ldr; e += GR_THREADS) {
            const int r = e / ldr, k = e % ldr;
            const bool in = r < rows && k < sk;
            const int64_t g = (jt + r) * sk + k;
            xs[e] = in ? X[g] : VT(0);
            ys[e] = in ? (Yadd ? fma(eta, Yadd[g], Y[g]) : Y[g]) : VT(0);
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < GR_TILES; ++t) {
            const int tile = threadIdx.x + t * GR_THREADS;
            if (tile < ntile) {
                const int a0 = (tile / ncg) * 4, c0 = (tile % ncg) * 4;
                for (int r = 0; r < rows; ++r) {
                    const TsVec4<VT> xa = *reinterpret_cast<const TsVec4<VT>*>(xs + r * ldr + a0);
                    const TsVec4<VT> yc = *reinterpret_cast<const TsVec4<VT>*>(ys + r * ldr + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[t][i][c] = fma(xa.v[i], yc.v[c], acc[t][i][c]);
                }
            }
        }
    }
    const int ss = sk * sk;
#pragma unroll
    for (int t = 0; t < GR_TILES; ++t) {
        const int tile = threadIdx.x + t * GR_THREADS;
        if (tile < ntile) {
            const int a0 = (tile / ncg) * 4, c0 = (tile % ncg) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (a0 + i < sk && c0 + c < sk)
                        part[(int64_t)blockIdx.x * ss + (a0 + i) * sk + c0 + c] = (double)acc[t][i][c];
        }
    }
}

// G[e] = sum over the nb partials, in block order (four interleaved running sums, combined in a
// fixed order: the result does not depend on the launch)
__global__ void gram_reduce(int nb, int ss, const double* part, double* G) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ss; e += gridDim.x * blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int b = 0;
        for (; b + 3 < nb; b += 4) {
            a0 += part[(int64_t)b * ss + e];
            a1 += part[(int64_t)(b + 1) * ss + e];
            a2 += part[(int64_t)(b + 2) * ss + e];
            a3 += part[(int64_t)(b + 3) * ss + e];
        }
        for (; b < nb; ++b) a0 += part[(int64_t)b * ss + e];
        G[e] = (a0 + a1) + (a2 + a3);
    }
}

// C (n x s) = X' (n x s) * Wm (s x s, value type), X' = X + eta Xadd when Xadd is given; in place
// (Cout == X) allowed: a block stages its tile of rows in shared memory before writing them.  Wm is
// staged once per block (rows padded to a multiple of 4 entries); each thread owns a 4 x 4 tile
// of the TS_ROWS x s output tile: per k, four broadcast loads of X' and one 4-wide load of Wm feed
// 16 FMAs.
constexpr int TS_THREADS = 256, TS_ROWS = 32;
template <typename VT>
static size_t ts_smem(int sk) {
    const size_t ldw = (size_t)((sk + 3) & ~3);
    return ((size_t)sk * ldw + (size_t)TS_ROWS * (sk + 1)) * sizeof(VT);
}
template <typename VT>
__global__ void __launch_bounds__(TS_THREADS) ts_gemm(int64_t n, int sk, const VT* X, const VT* Xadd,
                                                     const double* eta_p, const VT* Wm, VT* Cout) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const int ldw = (sk + 3) & ~3, ldx = sk + 1;
    VT* ws = reinterpret_cast<VT*>(tsm);   // sk x ldw
    VT* xs = ws + sk * ldw;                // TS_ROWS x ldx
    const VT eta = Xadd ? (VT)*eta_p : VT(0);
    for (int e = threadIdx.x; e < sk * ldw; e += TS_THREADS) {
        const int k = e / ldw, c = e % ldw;
        ws[e] = c < sk ? Wm[k * sk + c] : VT(0);
    }
    const int ncg = ldw / 4;
    const int rg = threadIdx.x / ncg, cg = threadIdx.x % ncg;
    const bool act = rg < TS_ROWS / 4;
    const int64_t ntile = (n + TS_ROWS - 1) / TS_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t j0 = tile * TS_ROWS;
        const int rows = (int)min((int64_t)TS_ROWS, n - j0);
        __syncthreads();   // Wm staged; the previous tile's reads are done
        for (int e = threadIdx.x; e < TS_ROWS * sk; e += TS_THREADS) {
            const int r = e / sk, k = e % sk;
            const int64_t g = (j0 + r) * sk + k;
            xs[r * ldx + k] = r < rows ? (Xadd ? fma(eta, Xadd[g], X[g]) : X[g]) : VT(0);
        }
        __syncthreads();
        if (act) {
            VT acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][c] = VT(0);
            const VT* xr = xs + (rg * 4) * ldx;
            for (int k = 0; k < sk; ++k) {
                const TsVec4<VT> w4 = *reinterpret_cast<const TsVec4<VT>*>(ws + k * ldw + cg * 4);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const VT xv = xr[i * ldx + k];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fma(xv, w4.v[c], acc[i][c]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = rg * 4 + i;
                if (r < rows) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (cg * 4 + c < sk) Cout[(j0 + r) * sk + cg * 4 + c] = acc[i][c];
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// One-CTA FP64 kernels on s x s matrices (s <= 256)
// ------------------------------------------------------------------------------------------
// In: G (s x s, symmetric part used).  Out: Cinv (value type, upper triangular inverse of the
// Cholesky factor C with G = C^T C); status[0] = 1 on success, 0 if G is not positive definite.
// Float64, one CTA, everything in shared memory: right-looking Cholesky, then the triangular
// inverse in place column by column (column j of C^{-1} is -C^{-1}[0:j,0:j] C[0:j,j] / c_jj,
// the rows of each column computed in parallel).
template <typename VT>
__global__ void __launch_bounds__(1024) chol_inv_kernel(int sk, const double* G, double* Cw, VT* Cinv,
                                                       int* status) {
    extern __shared__ __align__(16) unsigned char csm[];
    double* c = reinterpret_cast<double*>(csm);  // s x s
    double* tmp = c + sk * sk;                    // s
    __shared__ int ok;
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int i = e / sk, j = e % sk;
        c[e] = 0.5 * (G[i * sk + j] + G[j * sk + i]);
    }
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int k = 0; k < sk; ++k) {
        if (threadIdx.x == 0) {
            const double d = c[k * sk + k];
            if (!(d > 0.0)) ok = 0;
            c[k * sk + k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (!ok) break;
        const double piv = c[k * sk + k];
        for (int j = k + 1 + threadIdx.x; j < sk; j += blockDim.x) c[k * sk + j] /= piv;
        __syncthreads();
        const int rem = sk - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j >= i) c[i * sk + j] -= c[k * sk + i] * c[k * sk + j];
        }
        __syncthreads();
    }
    if (!ok) {
        if (threadIdx.x == 0) status[0] = 0;
        return;
    }
    for (int j = 0; j < sk; ++j) {
        for (int l = threadIdx.x; l < j; l += blockDim.x) tmp[l] = c[l * sk + j];
        __syncthreads();
        const double ajj = 1.0 / c[j * sk + j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            double acc = 0.0;
            for (int l = i; l < j; ++l) acc += c[i * sk + l] * tmp[l];
            c[i * sk + j] = -ajj * acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) c[j * sk + j] = ajj;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int i = e / sk, j = e % sk;
        Cinv[e] = (VT)(j >= i ? c[e] : 0.0);
    }
    (void)Cw;
    if (threadIdx.x == 0) status[0] = 1;
}

// The same factorisation and triangular inverse in float32 (float value types): G of the sketch
// is rounded to float, the right-looking Cholesky and the column-by-column inverse run in float
// arithmetic.  Float32 is about 64x the float64 rate of this part; the factor's backward error
// (~s eps32 ||G||) is far below the shift eta (= sqrt(n) eps32 ||Y||_F) for every sketch with a
// moderately conditioned core, and a non-positive pivot reports failure (status 0) so that the
// caller repeats the attempt in float64.
__global__ void __launch_bounds__(1024) chol_inv_f32_kernel(int sk, const double* G, float* Cinv, int* status) {
    extern __shared__ __align__(16) unsigned char csm[];
    float* c = reinterpret_cast<float*>(csm);  // s x s
    float* tmp = c + sk * sk;                  // s
    __shared__ int ok;
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int i = e / sk, j = e % sk;
        c[e] = (float)(0.5 * (G[i * sk + j] + G[j * sk + i]));
    }
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int k = 0; k < sk; ++k) {
        if (threadIdx.x == 0) {
            const float d = c[k * sk + k];
            if (!(d > 0.0f)) ok = 0;
            c[k * sk + k] = d > 0.0f ? sqrtf(d) : 1.0f;
        }
        __syncthreads();
        if (!ok) break;
        const float rpiv = 1.0f / c[k * sk + k];
        for (int j = k + 1 + threadIdx.x; j < sk; j += blockDim.x) c[k * sk + j] *= rpiv;
        __syncthreads();
        const int rem = sk - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j >= i) c[i * sk + j] = fmaf(-c[k * sk + i], c[k * sk + j], c[i * sk + j]);
        }
        __syncthreads();
    }
    if (!ok) {
        if (threadIdx.x == 0) status[0] = 0;
        return;
    }
    for (int j = 0; j < sk; ++j) {
        for (int l = threadIdx.x; l < j; l += blockDim.x) tmp[l] = c[l * sk + j];
        __syncthreads();
        const float ajj = 1.0f / c[j * sk + j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            float acc = 0.0f;
            for (int l = i; l < j; ++l) acc = fmaf(c[i * sk + l], tmp[l], acc);
            c[i * sk + j] = -ajj * acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) c[j * sk + j] = ajj;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int i = e / sk, j = e % sk;
        Cinv[e] = j >= i ? c[e] : 0.0f;
    }
    if (threadIdx.x == 0) status[0] = 1;
}

// Cyclic Jacobi eigendecomposition of the symmetric s x s matrix M (one CTA), arithmetic in T.
// Round-robin ("circle") ordering: in round r of a sweep over se = s + (s odd) indices, index
// se - 1 meets r and, for k = 1 .. se/2 - 1, (r + k) mod (se - 1) meets (r - k) mod (se - 1);
// the se/2 disjoint rotations of a round run in parallel (Golub & Van Loan §8.5).  A pair is
// rotated while |m_pq| > rot_tol sqrt(|m_pp m_qq|) (the relative test of Demmel & Veselic).  The
// iteration stops after a sweep in which no pair exceeded conv_tol = sqrt(rot_tol) at its turn:
// Jacobi converges quadratically, so that sweep already brought every pair to the rot_tol level
// (rotations at the arithmetic's noise never stop on their own).  V starts from Vinit (a warm start
// from a nearby problem, Min then being Vinit^T M Vinit) and from I otherwise, and accumulates
// the rotations.  Rows of M and V are stored with an odd stride so that the column updates
// are free of bank conflicts.  Out: Vout (s x s, columns = eigenvectors), ev (unsorted).
constexpr int JAC_MAX_PER_THREAD = 8;   // ceil((s/2) * s / 1024) for s <= 128
constexpr int JAC_MAX_BLK = 3;          // ceil((s/2) (s/2 + 1) / 2 / 1024) for s <= 128
template <typename T, bool VS>
__global__ void __launch_bounds__(1024) jacobi_kernel(int sk, const double* Min, const T* Vinit, T* Vout,
                                                     double* ev, int max_sweeps, double rot_tol,
                                                     int* sweeps_out) {
    extern __shared__ __align__(16) unsigned char jsm[];
    const int se = sk + (sk & 1);
    const int half = se / 2;
    const int ld = sk | 1;
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    T* M = reinterpret_cast<T*>(jsm);                   // s x ld
    T* Vs_ = M + sk * ld;                               // s x ld (VS only)
    // the round's rotations, one 8- or 16-byte load each: (c, s) and the pair p | q << 16
    T2* rot = reinterpret_cast<T2*>(
        (reinterpret_cast<uintptr_t>(VS ? Vs_ + sk * ld : Vs_) + 15) & ~static_cast<uintptr_t>(15));   // half
    int* pqs = reinterpret_cast<int*>(rot + half);      // half
    const int vld = VS ? ld : sk;
    T* V = VS ? Vs_ : Vout;
    __shared__ int nrot;
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int i = e / sk, j = e % sk;
        M[i * ld + j] = (T)(0.5 * (Min[i * sk + j] + Min[j * sk + i]));
        V[i * vld + j] = Vinit ? Vinit[e] : ((i == j) ? T(1) : T(0));
    }
    // this thread's (pair k, row i of V) work items, fixed for the whole iteration, packed as
    // k | (i * vld) << 16 (one register each: the kernel runs at the 64-register cap)
    int wkj[JAC_MAX_PER_THREAD];
    int nw = 0;
#pragma unroll
    for (int r = 0; r < JAC_MAX_PER_THREAD; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        wkj[r] = 0;
        if (e < half * sk) { wkj[r] = (e / sk) | (((e % sk) * vld) << 16); nw = r + 1; }
    }
    const T tol = (T)rot_tol;
    const T ctol = (T)sqrt(rot_tol);
    // float: the tests on squares (no square root) and the rotation from the fast reciprocal,
    // square root and division: this phase runs in two warps while the other thirty wait at the
    // barrier, so its latency is each round's; the rotation need not be exact (c^2 + s^2 = 1 to a
    // few ulp, and the polar step after the sweeps restores V's orthogonality)
    const float tol2 = (float)(rot_tol * rot_tol), ctol2 = (float)rot_tol;
    // this thread's pair blocks (a, b), b >= a, of the one-pass two-sided update, fixed for the
    // whole iteration (half (half + 1) / 2 <= 2080 blocks for s <= 128)
    int bab[JAC_MAX_BLK];   // a | b << 16
    int nb = 0;
    {
        int a = 0, rem = threadIdx.x;
        while (a < half && rem >= half - a) { rem -= half - a; ++a; }
#pragma unroll
        for (int r = 0; r < JAC_MAX_BLK; ++r) {
            bab[r] = 0;
            if (a < half) { bab[r] = a | ((a + rem) << 16); nb = r + 1; }
            // advance by blockDim.x blocks
            int step = blockDim.x;
            while (a < half && step > 0) {
                const int left = half - a - rem;   // blocks left in row a after this one
                if (step < left) { rem += step; step = 0; }
                else { step -= left; ++a; rem = 0; }
            }
        }
    }
    int sweep = 0;
    __syncthreads();
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) nrot = 0;
        __syncthreads();
        for (int round = 0; round < se - 1; ++round) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                // round-robin pairing: (round + k) and (round - k) mod (se - 1), with se - 1 last
                const int m1 = se - 1;
                int p, q;
                if (k == 0) { p = round; q = m1; }
                else {
                    p = round + k;
                    if (p >= m1) p -= m1;
                    q = round - k;
                    if (q < 0) q += m1;
                }
                if (p > q) { int t = p; p = q; q = t; }
                T c = T(1), s = T(0);
                if (q < sk) {
                    const T apq = M[p * ld + q];
                    const T app = M[p * ld + p], aqq = M[q * ld + q];
                    if constexpr (sizeof(T) == 4) {
                        const float a2 = apq * apq, pq = fabsf(app * aqq);
                        if (apq != 0.f && a2 > tol2 * pq) {
                            if (a2 > ctol2 * pq) nrot = 1;   // benign race: writers store 1
                            const float tau = __fdividef(aqq - app, 2.f * apq);
                            const float at = fabsf(tau);
                            // t = sign(tau) / (|tau| + sqrt(1 + tau^2)), about sign(tau) / (2 |tau|) for huge |tau|
                            float t = at < 1e18f ? __frcp_rn(at + __fsqrt_rn(fmaf(at, at, 1.f))) : __fdividef(0.5f, at);
                            t = tau >= 0.f ? t : -t;
                            c = rsqrtf(fmaf(t, t, 1.f));
                            s = t * c;
                        }
                    } else {
                        const T scale = sqrt(fabs(app * aqq));
                        if (apq != T(0) && fabs(apq) > tol * scale) {
                            if (fabs(apq) > ctol * scale) nrot = 1;   // benign race: writers store 1
                            const T tau = (aqq - app) / (T(2) * apq);
                            const T t = tau >= T(0) ? T(1) / (tau + sqrt(T(1) + tau * tau))
                                                    : T(-1) / (-tau + sqrt(T(1) + tau * tau));
                            c = T(1) / sqrt(T(1) + t * t);
                            s = t * c;
                        }
                    }
                }
                T2 cr;
                cr.x = c;
                cr.y = s;
                rot[k] = cr;
                pqs[k] = p | (q << 16);
            }
            __syncthreads();
            // M <- R M R^T in one pass: the 2 x 2 block of rows {p_a, q_a} and columns {p_b, q_b}
            // becomes R_a X R_b^T, with R_k = [[c_k, -s_k], [s_k, c_k]]; the blocks are disjoint,
            // so each is read and written by one thread (b >= a, mirrored: M stays symmetric)
#pragma unroll
            for (int r = 0; r < JAC_MAX_BLK; ++r) {
                if (r >= nb) break;
                const int a = bab[r] & 0xffff, bb = bab[r] >> 16;
                const T2 ra = rot[a], rb = rot[bb];
                const T sa = ra.y, sb = rb.y;
                if (sa == T(0) && sb == T(0)) continue;
                const T ca = ra.x, cb = rb.x;
                const int pqa = pqs[a], pqb = pqs[bb];
                const int pa = pqa & 0xffff, qa = pqa >> 16, pb = pqb & 0xffff, qb = pqb >> 16;
                const bool qa_ok = qa < sk, qb_ok = qb < sk;
                const T x00 = M[pa * ld + pb];
                const T x01 = qb_ok ? M[pa * ld + qb] : T(0);
                const T x10 = qa_ok ? M[qa * ld + pb] : T(0);
                const T x11 = (qa_ok && qb_ok) ? M[qa * ld + qb] : T(0);
                // T = R_a X
                const T t00 = ca * x00 - sa * x10, t01 = ca * x01 - sa * x11;
                const T t10 = sa * x00 + ca * x10, t11 = sa * x01 + ca * x11;
                // X' = T R_b^T
                const T y00 = t00 * cb - t01 * sb, y01 = t00 * sb + t01 * cb;
                const T y10 = t10 * cb - t11 * sb, y11 = t10 * sb + t11 * cb;
                M[pa * ld + pb] = y00;
                if (qb_ok) M[pa * ld + qb] = y01;
                if (qa_ok) M[qa * ld + pb] = y10;
                if (qa_ok && qb_ok) M[qa * ld + qb] = y11;
                if (a != bb) {
                    M[pb * ld + pa] = y00;
                    if (qb_ok) M[qb * ld + pa] = y01;
                    if (qa_ok) M[pb * ld + qa] = y10;
                    if (qa_ok && qb_ok) M[qb * ld + qa] = y11;
                }
            }
#pragma unroll
            for (int r = 0; r < JAC_MAX_PER_THREAD; ++r) {            // V <- V R^T
                if (r >= nw) break;
                const int k = wkj[r] & 0xffff, io = wkj[r] >> 16;
                const T2 rk = rot[k];
                const T sv = rk.y;
                if (sv == T(0)) continue;
                const int pqk = pqs[k];
                const int p = pqk & 0xffff, q = pqk >> 16;
                const T cv = rk.x;
                const T vp = V[io + p], vq = V[io + q];
                V[io + p] = cv * vp - sv * vq;
                V[io + q] = sv * vp + cv * vq;
            }
            __syncthreads();
        }
        const int any = nrot;
        __syncthreads();   // every thread has read nrot before thread 0 resets it
        if (any == 0) { ++sweep; break; }
    }
    if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
    for (int e = threadIdx.x; e < sk; e += blockDim.x) ev[e] = (double)M[e * ld + e];
    if (VS)
        for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) Vout[e] = V[(e / sk) * vld + e % sk];
}

// Warm start of the Jacobi iteration: Mout = V0^T M V0 for the s x s symmetric M and the
// eigenvector matrix V0 of a nearby matrix, in two passes (T1 = M V0, then V0^T T1).  One block
// per output row, value-type arithmetic.
template <typename T>
__global__ void congruence_kernel(int sk, int pass, const double* M, const T* V0, T* T1, double* Mout) {
    const int i = blockIdx.x;
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {
        T acc = T(0);
        if (pass == 0) {
            for (int k = 0; k < sk; ++k) acc += (T)M[i * sk + k] * V0[k * sk + c];
            T1[i * sk + c] = acc;
        } else {
            for (int k = 0; k < sk; ++k) acc += V0[k * sk + i] * T1[k * sk + c];
            Mout[i * sk + c] = (double)acc;
        }
    }
}

// One Newton-Schulz step towards the nearest orthogonal matrix, V <- V (3I - V^T V) / 2, which
// squares the orthogonality error of a V that is orthogonal up to rounding (the Jacobi rotations
// are applied in the value type, and warm starts would otherwise let that error accumulate from
// one sketch to the next).  pass 0: G = V^T V (float64 sums); pass 1: Vout = V (1.5 I - 0.5 G).
// One block per output row.
template <typename T>
__global__ void polar_step_kernel(int sk, int pass, const T* V, double* G, T* Vout) {
    const int i = blockIdx.x;
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {
        double acc = 0.0;
        if (pass == 0) {
            for (int k = 0; k < sk; ++k) acc += (double)V[k * sk + i] * (double)V[k * sk + c];
            G[i * sk + c] = acc;
        } else {
            for (int k = 0; k < sk; ++k) acc += (double)V[i * sk + k] * G[k * sk + c];
            Vout[i * sk + c] = (T)(1.5 * (double)V[i * sk + c] - 0.5 * acc);
        }
    }
}

// Float64 Rayleigh quotients ev_c = v_c^T M v_c / v_c^T v_c of the Jacobi eigenvectors against
// the float64 matrix M: the eigenvalue error becomes second order in the eigenvector error.
// One block per eigenpair.
template <typename T>
__global__ void eig_rq_kernel(int sk, const double* M, const T* V, double* ev) {
    const int c = blockIdx.x;
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < sk; i += blockDim.x) {
        double yi = 0.0;
        for (int k = 0; k < sk; ++k) yi += M[i * sk + k] * (double)V[k * sk + c];
        const double vi = (double)V[i * sk + c];
        num += vi * yi;
        den += vi * vi;
    }
    double a[2] = {num, den};
    block_sum<2>(a);
    if (threadIdx.x == 0) ev[c] = a[1] > 0.0 ? a[0] / a[1] : 0.0;
}

// Sort eigenpairs descending; Vs[k][c] = V[k][perm c] / sigma_c (value type);
// lam[c] = max(ev[perm c] - eta, 0).  One CTA.
template <typename VT, typename T>
__global__ void eig_finish_kernel(int sk, const T* V, const double* ev, const double* eta,
                                  VT* Vs, double* lam) {
    __shared__ int perm[256];
    __shared__ double sig[256];
    __shared__ double key[256];
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {
        const double e = ev[c];
        key[c] = e == e ? e : -INFINITY;   // NaN sorts last
    }
    __syncthreads();
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {   // rank sort, descending, stable
        const double kc = key[c];
        int rank = 0;
        for (int b = 0; b < sk; ++b) rank += (key[b] > kc || (key[b] == kc && b < c)) ? 1 : 0;
        perm[rank] = c;
    }
    __syncthreads();
    const double e0 = fmax(ev[perm[0]], 0.0);
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {
        const double e = ev[perm[c]];
        sig[c] = (e > 1e-30 * e0 && e > 0.0) ? sqrt(e) : 0.0;
        lam[c] = fmax(e - *eta, 0.0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < sk * sk; e += blockDim.x) {
        const int k = e / sk, c = e % sk;
        Vs[e] = sig[c] > 0.0 ? (VT)((double)V[k * sk + perm[c]] / sig[c]) : VT(0);
    }
}

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------
static size_t al(size_t b) { return (b + 255) & ~size_t(255); }
static int gram_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(128, n / 64)); }
static int ts_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(304, (n + TS_ROWS - 1) / TS_ROWS)); }

size_t nystrom_work_bytes(int prec, int64_t m, int64_t n, int sk) {
    const size_t vt = prec == P_FP64 ? 8 : 4;
    const size_t ss = (size_t)sk * sk;
    size_t b = 0;
    b += al(n * sk * vt);         // Oq
    b += al(m * sk * vt);         // W
    b += al(n * sk * vt);         // Y
    b += al(n * sk * vt);         // B (Y_eta, then B)
    b += al(ss * 8) * 3;          // G, C, M
    b += al(ss * vt);             // Cinv / Vs
    b += al(sk * 8);              // ev
    b += al(std::max<size_t>(gram_blocks(n) * ss, 1024) * 8);  // gpart
    b += al(64 * 8);              // scal
    b += al(64);                  // status
    b += al(ss * 8);              // V
    return b;
}

NysWork nystrom_carve(void* base, int prec, int64_t m, int64_t n, int sk) {
    const size_t vt = prec == P_FP64 ? 8 : 4;
    const size_t ss = (size_t)sk * sk;
    char* p = static_cast<char*>(base);
    NysWork w{};
    w.Oq = p; p += al(n * sk * vt);
    w.W = p; p += al(m * sk * vt);
    w.Y = p; p += al(n * sk * vt);
    w.B = p; p += al(n * sk * vt);
    w.G = reinterpret_cast<double*>(p); p += al(ss * 8);
    w.C = reinterpret_cast<double*>(p); p += al(ss * 8);
    w.M = reinterpret_cast<double*>(p); p += al(ss * 8);
    w.Cinv = p; p += al(ss * vt);
    w.ev = reinterpret_cast<double*>(p); p += al(sk * 8);
    w.gpart = reinterpret_cast<double*>(p); p += al(std::max<size_t>(gram_blocks(n) * ss, 1024) * 8);
    w.scal = reinterpret_cast<double*>(p); p += al(64 * 8);
    w.status = reinterpret_cast<int*>(p); p += al(64);
    // V shares the tail
    return w;
}

template <int P, typename VT>
static void launch_sketch(int64_t m, int64_t n, int sk, const void* A, int64_t lda,
                          const float* rs, const VT* d, const VT* Om, VT* W, VT* Y, cudaStream_t s) {
    dim3 g1((unsigned)((m + GT - 1) / GT), (unsigned)((sk + GT - 1) / GT));
    sketch_a_omega<P, VT><<<g1, 256, 0, s>>>(m, n, sk, A, lda, rs, d, Om, W);
    dim3 g2((unsigned)((n + GT - 1) / GT), (unsigned)((sk + GT - 1) / GT));
    sketch_at_w<P, VT><<<g2, 256, 0, s>>>(m, n, sk, A, lda, rs, W, Y);
    if (sync_check()) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) std::fprintf(stderr, "[genios] sketch: %s\n", cudaGetErrorString(e));
    }
}

// GENIOS_SYNC_CHECK=1 synchronises after every kernel of the core and reports the first
// failing one (diagnostics only; off by default).
static bool sync_check() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("GENIOS_SYNC_CHECK");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}
#define NYS_CHECK(name)                                                                     \
    do {                                                                                    \
        if (sync_check()) {                                                                 \
            cudaError_t _e = cudaStreamSynchronize(s);                                      \
            if (_e == cudaSuccess) _e = cudaGetLastError();                                 \
            if (_e != cudaSuccess) {                                                        \
                std::fprintf(stderr, "[genios] nystrom kernel %s: %s\n", name,              \
                             cudaGetErrorString(_e));                                       \
                return _e;                                                                  \
            }                                                                               \
        }                                                                                   \
    } while (0)

// Oq = orthonormal basis of range(Om) by CholeskyQR2: twice { G = Q^T Q (float64 sums);
// G = R^T R; Q <- Q R^{-1} }.  A Gaussian n x s matrix with s << n is well conditioned, so
// Cholesky QR is stable here and the second pass brings Q^T Q to the working precision.
template <typename VT>
static cudaError_t orthonormalize(int64_t n, int sk, const VT* Om, NysWork w, cudaStream_t s) {
    const int ss = sk * sk;
    const int gb = gram_blocks(n);
    const size_t gsm = gram_smem<VT>(sk);
    const size_t tsm = ts_smem<VT>(sk);
    const size_t csm = (size_t)ss * 8 + (size_t)sk * 8;
    {
        cudaError_t e = smem_optin<ts_gemm<VT>>();
        if (e == cudaSuccess) e = smem_optin<chol_inv_kernel<VT>>();
        if (e == cudaSuccess) e = smem_optin<gram_partial<VT>>();
        if (e != cudaSuccess) return e;
    }
    VT* Q = static_cast<VT*>(w.Oq);
    VT* Rinv = static_cast<VT*>(w.Cinv);
    const VT* src = Om;
    for (int pass = 0; pass < 2; ++pass) {
        gram_partial<VT><<<gb, GR_THREADS, gsm, s>>>(n, sk, src, src, nullptr, nullptr, 0.0, nullptr, w.gpart);
        gram_reduce<<<(ss + 255) / 256, 256, 0, s>>>(gb, ss, w.gpart, w.G);
        chol_inv_kernel<VT><<<1, 1024, csm, s>>>(sk, w.G, w.M, Rinv, w.status);
        NYS_CHECK("orthonormalize");
        ts_gemm<VT><<<ts_grid(n), TS_THREADS, tsm, s>>>(n, sk, src, nullptr, nullptr, Rinv, Q);
        NYS_CHECK("orthonormalize ts_gemm");
        src = Q;
    }
    return cudaGetLastError();
}

template <typename VT>
static cudaError_t core(int64_t n, int sk, const VT* Om, VT* Y, NysWork w, VT* U, double* lam,
                        double* eta_out, int* chol_ok, bool warm, cudaStream_t s) {
    const int64_t total = n * sk;
    const double eps = sizeof(VT) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
    double* fro2 = w.scal;
    double* eta = w.scal + 1;
    unsigned* counter = reinterpret_cast<unsigned*>(w.scal + 8);
    cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    // partials for the sum of squares reuse gpart (>= 1024 doubles as gram_blocks*ss >= s^2);
    // ||Y||_F^2 is read back together with the first Cholesky's status (one host sync)
    sumsq_kernel<VT><<<256, 256, 0, s>>>(total, Y, w.gpart, counter, fro2);
    NYS_CHECK("sumsq");
    const int ss = sk * sk;
    const int gb = gram_blocks(n);
    const size_t gsm = gram_smem<VT>(sk);
    const size_t tsm = ts_smem<VT>(sk);
    const size_t csm = (size_t)ss * 8 + (size_t)sk * 8;
    const int se = sk + (sk & 1);
    const size_t sld = (size_t)sk * (size_t)(sk | 1);
    const bool vs = 2 * sld * sizeof(VT) + (size_t)se * (sizeof(VT) + 4) <= 200 * 1024;
    const size_t jsm = (vs ? 2 : 1) * sld * sizeof(VT) + (size_t)se * (sizeof(VT) + 4) + 64;
    {
        cudaError_t e = smem_optin<ts_gemm<VT>>();
        if (e == cudaSuccess) e = smem_optin<chol_inv_kernel<VT>>();
        if (e == cudaSuccess) e = smem_optin<jacobi_kernel<VT, true>>();
        if (e == cudaSuccess) e = smem_optin<jacobi_kernel<VT, false>>();
        if (e == cudaSuccess) e = smem_optin<gram_partial<VT>>();
        if (e == cudaSuccess && sizeof(VT) == 4) e = smem_optin<chol_inv_f32_kernel>();
        if (e != cudaSuccess) return e;
    }
    VT* B = static_cast<VT*>(w.B);
    VT* Cinv = static_cast<VT*>(w.Cinv);
    double* V = w.C;  // reuse: C scratch holds eigenvectors after the Cholesky stage
    *chol_ok = 0;
    double mult = 1.0;
    const bool f32 = sizeof(VT) == 4;
    const size_t csm32 = (size_t)ss * 4 + (size_t)sk * 4;
    for (int attempt = 0; attempt < 7; ++attempt, mult *= 10.0) {
        // Omega^T Y_eta with Y_eta = Y + eta Omega, eta = sqrt(n) eps ||Y||_F mult (stored in eta)
        gram_partial<VT><<<gb, GR_THREADS, gsm, s>>>(n, sk, Om, Y, Om, fro2, std::sqrt((double)n) * eps * mult,
                                                     eta, w.gpart);
        NYS_CHECK("gram_partial(Omega, Y_eta)");
        gram_reduce<<<(ss + 255) / 256, 256, 0, s>>>(gb, ss, w.gpart, w.G);
        NYS_CHECK("gram_reduce");
        // float value types factor in float32 first, and in float64 only if that fails
        for (int dbl_pass = f32 ? 0 : 1; dbl_pass < 2; ++dbl_pass) {
            if (dbl_pass) chol_inv_kernel<VT><<<1, 1024, csm, s>>>(sk, w.G, w.M, Cinv, w.status);
            else chol_inv_f32_kernel<<<1, 1024, csm32, s>>>(sk, w.G, reinterpret_cast<float*>(Cinv), w.status);
            NYS_CHECK("chol_inv");
            struct { double f2; int st; } hv{0.0, 0};
            cudaMemcpyAsync(&hv.f2, fro2, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&hv.st, w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if (!std::isfinite(hv.f2)) {
                *chol_ok = -1;  // non-finite sketch
                return cudaSuccess;
            }
            if (hv.f2 == 0.0) {
                // A^T D A Omega = 0 (e.g. D = 0): the approximation is 0, lam = 0 and any
                // orthonormal U; Eq. (10) then reduces to the identity
                cudaMemcpyAsync(U, Om, (size_t)total * sizeof(VT), cudaMemcpyDeviceToDevice, s);
                cudaMemsetAsync(lam, 0, (size_t)sk * sizeof(double), s);
                if (eta_out) cudaMemsetAsync(eta_out, 0, sizeof(double), s);
                *chol_ok = 2;   // success without eigenvectors (nothing to warm-start from)
                return cudaGetLastError();
            }
            if (hv.st == 1) {
                *chol_ok = 1;
                break;
            }
        }
        if (*chol_ok) break;
    }
    if (!*chol_ok) return cudaSuccess;
    // B = Y_eta C^{-1}
    ts_gemm<VT><<<ts_grid(n), TS_THREADS, tsm, s>>>(n, sk, Y, Om, eta, Cinv, B);
    NYS_CHECK("ts_gemm(B)");
    // M = B^T B
    gram_partial<VT><<<gb, GR_THREADS, gsm, s>>>(n, sk, B, B, nullptr, nullptr, 0.0, nullptr, w.gpart);
    NYS_CHECK("gram_partial(B, B)");
    gram_reduce<<<(ss + 255) / 256, 256, 0, s>>>(gb, ss, w.gpart, w.M);
    NYS_CHECK("gram_reduce(M)");
    // Jacobi in the value type (a float64 Jacobi at s = 100 costs ~25 ms on this part's float64
    // pipe); in float32 the eigenvalues are then refined by float64 Rayleigh quotients
    VT* Vj = reinterpret_cast<VT*>(V);
    // relative pair tolerance near the arithmetic's resolution; a warm start (V of the previous
    // sketch of the same test matrix, which the slowly varying D leaves nearly diagonalising)
    // needs a few sweeps where a cold start needs about ten
    const int sweeps = sizeof(VT) == 8 ? 30 : 20;
    const double jtol = sizeof(VT) == 8 ? 1e-15 : 1e-7;
    const double* Mj = w.M;
    const VT* Vinit = nullptr;
    if (warm) {
        // Vj holds the previous eigenvectors; Cinv is free between ts_gemm(B) and eig_finish
        VT* T1 = Cinv;
        congruence_kernel<VT><<<sk, 128, 0, s>>>(sk, 0, w.M, Vj, T1, nullptr);
        congruence_kernel<VT><<<sk, 128, 0, s>>>(sk, 1, w.M, Vj, T1, w.G);
        NYS_CHECK("congruence");
        Mj = w.G;
        Vinit = Vj;
    }
    int* jsweeps = w.status + 1;
    if (vs) jacobi_kernel<VT, true><<<1, 1024, jsm, s>>>(sk, Mj, Vinit, Vj, w.ev, sweeps, jtol, jsweeps);
    else jacobi_kernel<VT, false><<<1, 1024, jsm, s>>>(sk, Mj, Vinit, Vj, w.ev, sweeps, jtol, jsweeps);
    NYS_CHECK("jacobi");
    polar_step_kernel<VT><<<sk, 128, 0, s>>>(sk, 0, Vj, w.G, nullptr);
    polar_step_kernel<VT><<<sk, 128, 0, s>>>(sk, 1, Vj, w.G, Cinv);
    cudaMemcpyAsync(Vj, Cinv, (size_t)ss * sizeof(VT), cudaMemcpyDeviceToDevice, s);
    NYS_CHECK("polar");
    if (sizeof(VT) == 4) {
        eig_rq_kernel<VT><<<sk, 128, 0, s>>>(sk, w.M, Vj, w.ev);
        NYS_CHECK("eig_rq");
    }
    eig_finish_kernel<VT, VT><<<1, 256, 0, s>>>(sk, Vj, w.ev, eta, Cinv, lam);
    NYS_CHECK("eig_finish");
    // U = B V Sigma^{-1}
    ts_gemm<VT><<<ts_grid(n), TS_THREADS, tsm, s>>>(n, sk, B, nullptr, nullptr, Cinv, U);
    NYS_CHECK("ts_gemm(U)");
    if (eta_out) cudaMemcpyAsync(eta_out, eta, sizeof(double), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

cudaError_t nystrom_build(int prec, int64_t m, int64_t n, int sk, const void* A, int64_t lda,
                          const float* rs, const void* d, const void* Om, void* U, double* lam,
                          double* eta_out, NysWork w, int* chol_ok, int flags, const TcSketch* tc,
                          cudaStream_t s) {
    if (sk < 1 || sk > 128) return cudaErrorInvalidValue;
    const bool reuse = (flags & NYS_REUSE_BASIS) != 0;
    const bool warm = (flags & NYS_WARM_EIG) != 0;
    if (prec == P_FP64) {
        if (!reuse) {
            cudaError_t e = orthonormalize<double>(n, sk, static_cast<const double*>(Om), w, s);
            if (e != cudaSuccess) return e;
        }
        const double* Oq = static_cast<const double*>(w.Oq);
        launch_sketch<P_FP64, double>(m, n, sk, A, lda, rs, static_cast<const double*>(d), Oq,
                                      static_cast<double*>(w.W), static_cast<double*>(w.Y), s);
        return core<double>(n, sk, Oq, static_cast<double*>(w.Y), w, static_cast<double*>(U), lam,
                            eta_out, chol_ok, warm, s);
    }
    const float* df = static_cast<const float*>(d);
    if (!reuse) {
        cudaError_t e = orthonormalize<float>(n, sk, static_cast<const float*>(Om), w, s);
        if (e != cudaSuccess) return e;
        if (tc) {   // the basis is rounded to the bf16 values the tensor cores multiply
            e = tc_pack_omega(tc->plan, tc->work, static_cast<float*>(w.Oq), s);
            if (e != cudaSuccess) return e;
        }
    }
    const float* Of = static_cast<const float*>(w.Oq);
    float* Wf = static_cast<float*>(w.W);
    float* Yf = static_cast<float*>(w.Y);
    if (tc) {
        cudaError_t e = cudaMemsetAsync(tc->work.err, 0, sizeof(int), s);
        if (e == cudaSuccess) e = tc_sketch(tc->plan, tc->work, df, Yf, tc->wait_limit, s);
        int err = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, tc->work.err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (err != 0) {   // a bounded wait of the tensor-core products ran out: Y is incomplete
            *chol_ok = -2;
            return cudaSuccess;
        }
        return core<float>(n, sk, Of, Yf, w, static_cast<float*>(U), lam, eta_out, chol_ok, warm, s);
    }
    if (prec == P_FP32) launch_sketch<P_FP32, float>(m, n, sk, A, lda, rs, df, Of, Wf, Yf, s);
    else if (prec == P_BF16) launch_sketch<P_BF16, float>(m, n, sk, A, lda, rs, df, Of, Wf, Yf, s);
    else if (prec == P_FP8) launch_sketch<P_FP8, float>(m, n, sk, A, lda, rs, df, Of, Wf, Yf, s);
    else return cudaErrorInvalidValue;
    return core<float>(n, sk, Of, Yf, w, static_cast<float*>(U), lam, eta_out, chol_ok, warm, s);
}

// ------------------------------------------------------------------------------------------
// Quantisation of a float32 matrix (setup)
// ------------------------------------------------------------------------------------------
__global__ void bf16_hilo_kernel(int64_t m, int64_t n, const float* A, int64_t ldi,
                                 __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo) {
    const int64_t total = m * ldo;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldo, j = e % ldo;
        const float a = j < n ? A[i * ldi + j] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(a);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(a - __bfloat162float(h));
    }
}

__global__ void fp8_rows_kernel(int64_t m, int64_t n, const float* A, int64_t ldi, uint8_t* q,
                                float* scale, int64_t ldo) {
    __shared__ float red[32];
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        float mx = 0.0f;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(A[i * ldi + j]));
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x < 32) {
            float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
            t = warp_max(t);
            if (threadIdx.x == 0) red[0] = t;
        }
        __syncthreads();
        const float amax = red[0];
        float sc = __fdiv_rn(amax, 448.0f);
        if (sc == 0.0f) sc = 1.0f;
        if (threadIdx.x == 0) scale[i] = sc;
        for (int64_t j = threadIdx.x; j < ldo; j += blockDim.x) {
            uint8_t code = 0;
            if (j < n) {
                const float v = __fdiv_rn(A[i * ldi + j], sc);
                code = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
            }
            q[i * ldo + j] = code;
        }
        __syncthreads();
    }
}

cudaError_t quantize_bf16_hilo(int64_t m, int64_t n, const float* A, int64_t lda_in, void* hi,
                               void* lo, int64_t lda_out, cudaStream_t s) {
    const int64_t total = m * lda_out;
    int grid = (int)std::min<int64_t>(152 * 32, (total + 255) / 256);
    if (grid < 1) grid = 1;
    bf16_hilo_kernel<<<grid, 256, 0, s>>>(m, n, A, lda_in, static_cast<__nv_bfloat16*>(hi),
                                          static_cast<__nv_bfloat16*>(lo), lda_out);
    return cudaGetLastError();
}

cudaError_t quantize_fp8_rows(int64_t m, int64_t n, const float* A, int64_t lda_in, uint8_t* q,
                              float* scale, int64_t lda_out, cudaStream_t s) {
    int grid = (int)std::min<int64_t>(152 * 16, m);
    if (grid < 1) grid = 1;
    fp8_rows_kernel<<<grid, 256, 0, s>>>(m, n, A, lda_in, q, scale, lda_out);
    return cudaGetLastError();
}

}  // namespace genios

// ------------------------------------------------------------------------------------------
// Adaptive sketch size (§2.2): power-method steps on E = H_data - U diag(lam) U^T
// ------------------------------------------------------------------------------------------
namespace genios {

constexpr int NYS_ROWS = 64;   // rows of U per block of the U^T v partials

// block partials of U^T v over NYS_ROWS rows: part[b][c], c < 128 (threads: c = t % 128, two halves)
template <typename VT>
__global__ void nys_utv_part_kernel(int64_t n, int sk, const VT* U, const VT* v, double* part) {
    __shared__ double sh[256];
    const int t = threadIdx.x, c = t & 127, h = t >> 7;
    const int64_t r0 = (int64_t)blockIdx.x * NYS_ROWS;
    double acc = 0.0;
    if (c < sk)
        for (int r = h; r < NYS_ROWS; r += 2) {
            const int64_t j = r0 + r;
            if (j < n) acc += (double)U[j * sk + c] * (double)v[j];
        }
    sh[t] = acc;
    __syncthreads();
    if (t < 128) part[(size_t)blockIdx.x * 128 + t] = c < sk ? sh[t] + sh[t + 128] : 0.0;
}

// w_c = lam_c sum_b part[b][c], in block order
__global__ void nys_utv_reduce_kernel(int nb, int sk, const double* part, const double* lam, double* w) {
    const int c = threadIdx.x;
    if (c >= 128) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * 128 + c];
    w[c] = c < sk ? lam[c] * s : 0.0;
}

// y -= U w, and out = [v^T y, y^T y, v^T v]
template <typename VT>
__global__ void nys_err_apply_kernel(int64_t n, int sk, const VT* U, const double* w, const VT* v, VT* y,
                                     Scratch sc, double* out) {
    __shared__ double wsh[128];
    for (int c = threadIdx.x; c < 128; c += blockDim.x) wsh[c] = w[c];
    __syncthreads();
    double d[3] = {0.0, 0.0, 0.0};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < sk; ++c) acc += (double)U[j * sk + c] * wsh[c];
        const double yj = (double)y[j] - acc;
        y[j] = (VT)yj;
        const double vj = (double)v[j];
        d[0] += vj * yj;
        d[1] += yj * yj;
        d[2] += vj * vj;
    }
    double o[3];
    if (grid_sum<3>(d, sc.part, sc.counter, o) && threadIdx.x == 0) {
        out[0] = o[0];
        out[1] = o[1];
        out[2] = o[2];
    }
}

template <typename VT>
__global__ void nys_scale_kernel(int64_t n, const VT* y, double scale, VT* v) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        v[j] = (VT)((double)y[j] * scale);
}

template <typename VT>
static cudaError_t err_step_vt(int64_t n, int sk, const void* U, const double* lam, const void* v, void* y,
                               double* out3, Scratch sc, cudaStream_t s) {
    const int nb = (int)((n + NYS_ROWS - 1) / NYS_ROWS);
    double* part = sc.part + 65536;
    double* w = part + (size_t)nb * 128;
    nys_utv_part_kernel<VT><<<nb, 256, 0, s>>>(n, sk, static_cast<const VT*>(U), static_cast<const VT*>(v), part);
    nys_utv_reduce_kernel<<<1, 128, 0, s>>>(nb, sk, part, lam, w);
    const int g = (int)std::min<int64_t>(256, (n + 255) / 256);
    nys_err_apply_kernel<VT><<<g, 256, 0, s>>>(n, sk, static_cast<const VT*>(U), w, static_cast<const VT*>(v),
                                               static_cast<VT*>(y), sc, out3);
    return cudaGetLastError();
}

cudaError_t nys_error_step(bool dbl, int64_t n, int sk, const void* U, const double* lam, const void* v, void* y,
                           double* out3, Scratch sc, cudaStream_t s) {
    if (sk < 0 || sk > 128 || (size_t)((n + NYS_ROWS - 1) / NYS_ROWS) * 128 + 128 > 196608) return cudaErrorInvalidValue;
    return dbl ? err_step_vt<double>(n, sk, U, lam, v, y, out3, sc, s)
               : err_step_vt<float>(n, sk, U, lam, v, y, out3, sc, s);
}

cudaError_t nys_scale(bool dbl, int64_t n, const void* y, double scale, void* v, cudaStream_t s) {
    const int g = (int)std::min<int64_t>(512, (n + 255) / 256);
    if (dbl) nys_scale_kernel<double><<<g, 256, 0, s>>>(n, static_cast<const double*>(y), scale, static_cast<double*>(v));
    else nys_scale_kernel<float><<<g, 256, 0, s>>>(n, static_cast<const float*>(y), scale, static_cast<float*>(v));
    return cudaGetLastError();
}

}  // namespace genios
