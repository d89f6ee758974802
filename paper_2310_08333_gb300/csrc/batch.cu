// Lockstep solve of K problems that share one data set (squared loss, float32): a
// regularisation path min_x 1/2||A x - b||^2 + lam1_k ||x||_1 + lam2_k/2 ||x||^2, k = 1..K,
// with every ADMM iteration (§2, Eqs. (3)-(5)) and every CG step (§2.1) taken for all K at once.
//
// The Hessian is the same for all K (A^T A; D = I for the squared loss, §3.3), so one product
// serves the whole batch: Y = A^T (A P) for the n x K matrix P of search directions runs as two
// tensor-core GEMMs (umma.cu) that read A once each, instead of K matrix-vector passes.
//   * CG products: bf16 A (the inexact Hessian the method allows, reading R2) with P split into
//     bf16 hi + lo, so the only rounding is that of A.
//   * Gradients (ADMM, stop tests): A split into bf16 hi + lo as well (two more GEMMs), about
//     2^-16 relative, the accuracy of the split-BF16 gradient of the mixed mode.
// One Nystrom sketch of A^T A serves every problem; the preconditioner coefficients of
// Eq. (10) use each problem's nu_k.  Vectors are n x K column-major; the per-problem vector
// work runs on grids of (row blocks) x K with per-problem reductions, and the preconditioner's
// U^T R and U C products stage U in shared memory once per row block for all K columns.
#include "common.cuh"
#include "internal.h"
#include "genios.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace genios {

constexpr int BK_T = 256;        // threads of the column-wise kernels
constexpr int BK_RB = 256;       // rows per block of the column-wise kernels
constexpr int BK_NV = 8;         // reduced values per column and block

struct BState {                  // per problem (device array of K)
    double rho, nu, lam1, lam2, u_scale, tol;
    double rhs2, rr, rz, pq, alpha, beta;
    double rd2, rhou2, rp2, x2, z2, u2, nnz, kd2, kg2;
    int active, cg_active, cg_it, cg_max;
};

// ------------------------------------------------------------------------------------------
// operand packing for the multi-RHS products
// ------------------------------------------------------------------------------------------
GENIOS_DEV uint4 bpack8(const float (&v)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i])) |
               ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i + 1])) << 16);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// P (n x K column-major, ld ldn) -> N-side operand of 2 Kp rows: rows c < Kp hold bf16(P[:, c]),
// rows Kp + c the remainders bf16(P - bf16(P)); k runs over the n features.
__global__ void bk_pack_p_kernel(int64_t n, int K, int Kp, int64_t ldn, const float* P, int64_t kpad,
                                 unsigned char* out) {
    const int64_t kch = kpad / 8, total = (int64_t)Kp * kch;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / kch);
        const int64_t j0 = (e % kch) * 8;
        float hi[8], lo[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float x = (c < K && j0 + t < n) ? P[(int64_t)c * ldn + j0 + t] : 0.0f;
            const float h = __bfloat162float(__float2bfloat16_rn(x));
            hi[t] = h;
            lo[t] = x - h;
        }
        *reinterpret_cast<uint4*>(out + blk_off(c, j0, kpad / 64, 2 * Kp)) = bpack8(hi);
        *reinterpret_cast<uint4*>(out + blk_off(Kp + c, j0, kpad / 64, 2 * Kp)) = bpack8(lo);
    }
}

// W = sum over splits and over the hi / lo column halves (and over the A hi / lo products when
// part_b is given) of the first product, packed hi + lo as the N-side operand of the second.
__global__ void bk_finish_w_kernel(int64_t m, int K, int Kp, const float* part_a, const float* part_b, int splits,
                                   int64_t mrows, int64_t kpad, unsigned char* out) {
    const int64_t kch = kpad / 8, total = (int64_t)Kp * kch;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / kch);
        const int64_t i0 = (e % kch) * 8;
        float hi[8], lo[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int64_t i = i0 + t;
            float w = 0.0f;
            if (c < K && i < m) {
                for (int z = 0; z < splits; ++z) {
                    const float* ra = part_a + ((int64_t)z * mrows + i) * (2 * Kp);
                    w += ra[c] + ra[Kp + c];
                    if (part_b) {
                        const float* rb = part_b + ((int64_t)z * mrows + i) * (2 * Kp);
                        w += rb[c] + rb[Kp + c];
                    }
                }
            }
            const float h = __bfloat162float(__float2bfloat16_rn(w));
            hi[t] = h;
            lo[t] = w - h;
        }
        *reinterpret_cast<uint4*>(out + blk_off(c, i0, kpad / 64, 2 * Kp)) = bpack8(hi);
        *reinterpret_cast<uint4*>(out + blk_off(Kp + c, i0, kpad / 64, 2 * Kp)) = bpack8(lo);
    }
}

// Y (n x K column-major) = sum over splits, column halves and A hi / lo of the second product
__global__ void bk_finish_y_kernel(int64_t n, int K, int Kp, const float* part_a, const float* part_b, int splits,
                                   int64_t nrows, int64_t ldn, float* Y) {
    const int64_t total = n * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % K);
        const int64_t j = e / K;
        float y = 0.0f;
        for (int z = 0; z < splits; ++z) {
            const float* ra = part_a + ((int64_t)z * nrows + j) * (2 * Kp);
            y += ra[c] + ra[Kp + c];
            if (part_b) {
                const float* rb = part_b + ((int64_t)z * nrows + j) * (2 * Kp);
                y += rb[c] + rb[Kp + c];
            }
        }
        Y[(int64_t)c * ldn + j] = y;
    }
}

// ------------------------------------------------------------------------------------------
// column-wise vector kernels: grid (row blocks, K); partials part[(k nb + b) BK_NV + v]
// ------------------------------------------------------------------------------------------
template <int NV>
GENIOS_DEV void col_partials(float (&v)[NV], double* part) {
    __shared__ float sh[NV][BK_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q][wid] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < BK_T / 32; ++w) s += sh[threadIdx.x][w];
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * BK_NV + threadIdx.x] = (double)s;
    }
}

#define BK_ROW_LOOP                                                       \
    const int k = blockIdx.y;                                             \
    const int64_t j = (int64_t)blockIdx.x * BK_RB + threadIdx.x;          \
    const bool in = j < n;                                                \
    const int64_t o = (int64_t)k * ldn + j

// G = Y + g0 + lam2 X (g0 = A^T l'(-b) = -A^T b); partials ||G + rho U||^2, ||rho U||^2
__global__ void bk_grad_kernel(int64_t n, int64_t ldn, const float* Y, const float* g0, const float* X, const float* U,
                               const BState* BS, float* G, double* part) {
    BK_ROW_LOOP;
    float v[2] = {0.f, 0.f};
    if (in && BS[k].active) {
        const float g = Y[o] + g0[j] + (float)BS[k].lam2 * X[o];
        G[o] = g;
        const float ru = (float)BS[k].rho * U[o];
        v[0] = (g + ru) * (g + ru);
        v[1] = ru * ru;
    }
    col_partials<2>(v, part);
}

// U <- u_scale U; R = -(G + rho (X - Z + U)); Delta = 0; partial ||R||^2
__global__ void bk_rhs_kernel(int64_t n, int64_t ldn, const float* G, const float* X, const float* Z, float* U,
                              const BState* BS, float* R, float* Dl, double* part) {
    BK_ROW_LOOP;
    float v[1] = {0.f};
    if (in && BS[k].active) {
        const float u = U[o] * (float)BS[k].u_scale;
        U[o] = u;
        const float r = -(G[o] + (float)BS[k].rho * (X[o] - Z[o] + u));
        R[o] = r;
        Dl[o] = 0.0f;
        v[0] = r * r;
    }
    col_partials<1>(v, part);
}

// Q = Qraw + nu P; partial p^T q
__global__ void bk_q_kernel(int64_t n, int64_t ldn, const float* Qraw, const float* P, const BState* BS, float* Q,
                            double* part) {
    BK_ROW_LOOP;
    float v[1] = {0.f};
    if (in && BS[k].cg_active) {
        const float p = P[o];
        const float q = Qraw[o] + (float)BS[k].nu * p;
        Q[o] = q;
        v[0] = p * q;
    }
    col_partials<1>(v, part);
}

// Delta += alpha P; R -= alpha Q; partial ||R||^2
__global__ void bk_upd_kernel(int64_t n, int64_t ldn, const float* P, const float* Q, const BState* BS, float* R,
                              float* Dl, double* part) {
    BK_ROW_LOOP;
    float v[1] = {0.f};
    if (in && BS[k].cg_active) {
        const float a = (float)BS[k].alpha;
        Dl[o] += a * P[o];
        const float r = R[o] - a * Q[o];
        R[o] = r;
        v[0] = r * r;
    }
    col_partials<1>(v, part);
}

// x += delta; x^ = alpha x + (1 - alpha) z; z = S(x^ + u, lam1 / rho); u += x^ - z (§2.5, §3.1,
// Eq. (5)); partials ||x - z||^2, ||x||^2, ||z||^2, ||rho u||^2, nnz(z)
__global__ void bk_zu_kernel(int64_t n, int64_t ldn, const float* Dl, float* X, float* Z, float* U, double over,
                             const BState* BS, double* part) {
    BK_ROW_LOOP;
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (in && BS[k].active) {
        const float x = X[o] + Dl[o];
        X[o] = x;
        const float zo = Z[o];
        const float xh = (float)over * x + (1.0f - (float)over) * zo;
        const float kap = (float)(BS[k].lam1 / BS[k].rho);
        const float t = xh + U[o];
        const float zn = t > kap ? t - kap : (t < -kap ? t + kap : 0.0f);
        Z[o] = zn;
        const float un = U[o] + xh - zn;
        U[o] = un;
        const float ru = (float)BS[k].rho * un;
        v[0] = (x - zn) * (x - zn);
        v[1] = x * x;
        v[2] = zn * zn;
        v[3] = ru * ru;
        v[4] = zn != 0.0f ? 1.0f : 0.0f;
    }
    col_partials<5>(v, part);
}

// relative KKT at z (reading R6): Gz = Yz + g0 + lam2 z; partials ||dist(0, dF(z))||^2, ||Gz||^2
__global__ void bk_kkt_kernel(int64_t n, int64_t ldn, const float* Yz, const float* g0, const float* Z,
                              const BState* BS, double* part) {
    BK_ROW_LOOP;
    float v[2] = {0.f, 0.f};
    if (in && BS[k].active) {
        const float z = Z[o];
        const float g = Yz[o] + g0[j] + (float)BS[k].lam2 * z;
        const float l1 = (float)BS[k].lam1;
        float d;
        if (z > 0.0f) d = fabsf(g + l1);
        else if (z < 0.0f) d = fabsf(g - l1);
        else d = fmaxf(fabsf(g) - l1, 0.0f);
        v[0] = d * d;
        v[1] = g * g;
    }
    col_partials<2>(v, part);
}

// U^T R block partials: block b covers rows [b URB, (b+1) URB) for every column;
// part_w[(b K + k) s + c]
__global__ void bk_ut_kernel(int64_t n, int64_t ldn, int K, int sk, int urb, const float* Un, const float* R,
                             double* part_w) {
    extern __shared__ float ush[];
    float* Us = ush;                        // urb x sk
    float* Rs = ush + (size_t)urb * sk;     // K x urb
    const int64_t j0 = (int64_t)blockIdx.x * urb;
    const int rows = (int)min((int64_t)urb, n - j0);
    for (int e = threadIdx.x; e < urb * sk; e += blockDim.x) {
        const int i = e / sk;
        Us[e] = i < rows ? Un[(j0 + i) * sk + e % sk] : 0.0f;
    }
    for (int e = threadIdx.x; e < K * urb; e += blockDim.x) {
        const int k = e / urb, i = e % urb;
        Rs[e] = i < rows ? R[(int64_t)k * ldn + j0 + i] : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * sk; e += blockDim.x) {
        const int k = e / sk, c = e % sk;
        float a0 = 0.0f, a1 = 0.0f;
        int i = 0;
        for (; i + 1 < rows; i += 2) {
            a0 = fmaf(Us[i * sk + c], Rs[k * urb + i], a0);
            a1 = fmaf(Us[(i + 1) * sk + c], Rs[k * urb + i + 1], a1);
        }
        if (i < rows) a0 = fmaf(Us[i * sk + c], Rs[k * urb + i], a0);
        part_w[((size_t)blockIdx.x * K + k) * sk + c] = (double)(a0 + a1);
    }
}

// Zc = R + U C_k (C = K x sk coefficients); P = Zc + beta_k P (start: P = Zc)
__global__ void bk_uc_kernel(int64_t n, int64_t ldn, int K, int sk, int urb, const float* Un, const float* R,
                             const float* Cw, const BState* BS, int start, float* P) {
    extern __shared__ float ush[];
    float* Us = ush;                      // urb x sk
    float* Cs = ush + (size_t)urb * sk;   // K x sk
    const int64_t j0 = (int64_t)blockIdx.x * urb;
    const int rows = (int)min((int64_t)urb, n - j0);
    for (int e = threadIdx.x; e < urb * sk; e += blockDim.x) {
        const int i = e / sk;
        Us[e] = i < rows ? Un[(j0 + i) * sk + e % sk] : 0.0f;
    }
    for (int e = threadIdx.x; e < K * sk; e += blockDim.x) Cs[e] = Cw[e];
    __syncthreads();
    for (int e = threadIdx.x; e < K * urb; e += blockDim.x) {
        const int k = e / urb, i = e % urb;
        if (i >= rows || !BS[k].cg_active) continue;
        float acc = 0.0f;
        for (int c = 0; c < sk; ++c) acc = fmaf(Us[i * sk + c], Cs[k * sk + c], acc);
        const int64_t o = (int64_t)k * ldn + j0 + i;
        const float zc = R[o] + acc;
        P[o] = start ? zc : zc + (float)BS[k].beta * P[o];
    }
}

// ------------------------------------------------------------------------------------------
// per-problem reductions and scalar logic: one block per problem
// ------------------------------------------------------------------------------------------
enum { RED_GRAD = 0, RED_RHS, RED_Q, RED_UPD, RED_ZU, RED_KKT };

__global__ void bk_reduce_kernel(int mode, int nb, const double* part, BState* BS) {
    const int k = blockIdx.x;
    double v[BK_NV];
#pragma unroll
    for (int q = 0; q < BK_NV; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < BK_NV; ++q) v[q] += part[((size_t)k * nb + b) * BK_NV + q];
    block_sum<BK_NV>(v);
    if (threadIdx.x != 0) return;
    BState& s = BS[k];
    switch (mode) {
        case RED_GRAD: s.rd2 = v[0]; s.rhou2 = v[1]; break;
        case RED_RHS:
            s.rhs2 = v[0];
            s.rr = v[0];
            s.cg_it = 0;
            s.cg_active = (s.active && v[0] > 0.0) ? 1 : 0;
            break;
        case RED_Q:
            if (s.cg_active) {
                s.pq = v[0];
                s.alpha = v[0] > 0.0 ? s.rz / v[0] : 0.0;
            } else {
                s.alpha = 0.0;
            }
            break;
        case RED_UPD: if (s.cg_active) s.rr = v[0]; break;
        case RED_ZU: if (s.active) { s.rp2 = v[0]; s.x2 = v[1]; s.z2 = v[2]; s.u2 = v[3]; s.nnz = v[4]; } break;
        case RED_KKT: if (s.active) { s.kd2 = v[0]; s.kg2 = v[1]; } break;
    }
}

// w = U^T R (reduce the block partials), C = ((lam_s + nu_k) / (lam_i + nu_k) - 1) w (Eq. (10)),
// r^T z = ||r||^2 + C^T w, beta, stop test.  One block per problem.
__global__ void bk_w_kernel(int start, int nbu, int K, int sk, const double* part_w, const double* lam, BState* BS,
                            float* Cw) {
    const int k = blockIdx.x;
    BState& s = BS[k];
    const double ls = lam[sk - 1];
    const double nu = s.nu;
    double loc = 0.0;
    for (int c = threadIdx.x; c < sk; c += blockDim.x) {
        double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        int b = 0;
        for (; b + 3 < nbu; b += 4) {
            w0 += part_w[((size_t)b * K + k) * sk + c];
            w1 += part_w[((size_t)(b + 1) * K + k) * sk + c];
            w2 += part_w[((size_t)(b + 2) * K + k) * sk + c];
            w3 += part_w[((size_t)(b + 3) * K + k) * sk + c];
        }
        for (; b < nbu; ++b) w0 += part_w[((size_t)b * K + k) * sk + c];
        const double w = (w0 + w1) + (w2 + w3);
        const double cw = ((ls + nu) / (lam[c] + nu) - 1.0) * w;
        Cw[k * sk + c] = (float)cw;
        loc += cw * w;
    }
    double v[1] = {loc};
    block_sum<1>(v);
    if (threadIdx.x != 0) return;
    if (!s.cg_active) return;
    const double rz = s.rr + v[0];
    if (start) {
        s.beta = 0.0;
    } else {
        s.beta = s.rz > 0.0 ? rz / s.rz : 0.0;
        s.cg_it += 1;
        if (!(s.pq > 0.0) || s.rr <= s.tol * s.tol * s.rhs2 || s.cg_it >= s.cg_max) s.cg_active = 0;
    }
    s.rz = rz;
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
namespace {

int64_t rup(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

struct Buf {
    std::vector<void*> ptrs;
    cudaError_t get(void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Buf() {
        for (void* p : ptrs) cudaFree(p);
    }
};

struct Ctx {
    int64_t m, n, ldn;
    int K, Kp, sk;
    int64_t rpad_m, kpad_n, rpad_n, kpad_m;
    int s1, s2;
    unsigned char *Ah_rows, *Al_rows, *Ah_cols, *Al_cols, *Bx, *Bw;
    float *part1a, *part1b, *part2a, *part2b;
    int* err;
    long long wait;
    cudaStream_t s;
};

// Y = A^T A X for the n x K matrix X: accurate (A hi + lo) or with bf16 A (CG products)
cudaError_t ata(const Ctx& c, const float* X, float* Y, bool accurate) {
    const int G = 4 * tc_sm_count();
    bk_pack_p_kernel<<<G, 256, 0, c.s>>>(c.n, c.K, c.Kp, c.ldn, X, c.kpad_n, c.Bx);
    cudaError_t e = tc_gemm(c.Ah_rows, c.Bx, c.part1a, c.rpad_m / 128, c.kpad_n / 64, 2 * c.Kp, c.s1, c.err, c.wait, c.s);
    if (e == cudaSuccess && accurate)
        e = tc_gemm(c.Al_rows, c.Bx, c.part1b, c.rpad_m / 128, c.kpad_n / 64, 2 * c.Kp, c.s1, c.err, c.wait, c.s);
    if (e != cudaSuccess) return e;
    bk_finish_w_kernel<<<G, 256, 0, c.s>>>(c.m, c.K, c.Kp, c.part1a, accurate ? c.part1b : nullptr, c.s1, c.rpad_m,
                                           c.kpad_m, c.Bw);
    e = tc_gemm(c.Ah_cols, c.Bw, c.part2a, c.rpad_n / 128, c.kpad_m / 64, 2 * c.Kp, c.s2, c.err, c.wait, c.s);
    if (e == cudaSuccess && accurate)
        e = tc_gemm(c.Al_cols, c.Bw, c.part2b, c.rpad_n / 128, c.kpad_m / 64, 2 * c.Kp, c.s2, c.err, c.wait, c.s);
    if (e != cudaSuccess) return e;
    bk_finish_y_kernel<<<G, 256, 0, c.s>>>(c.n, c.K, c.Kp, c.part2a, accurate ? c.part2b : nullptr, c.s2, c.rpad_n,
                                           c.ldn, Y);
    return cudaGetLastError();
}

}  // namespace

cudaError_t batch_pack_lo(const TcPlan& p, TcWork w, const float* A, int64_t lda, cudaStream_t s);

BatchResult batch_path_solve(const BatchInput& in, std::vector<::genios_info>& info) {
    BatchResult res{};
    res.status = GENIOS_OK;
    const int64_t m = in.m, n = in.n;
    const int K = in.K;
    if (K < 1 || K > 128 || in.sk < 1 || in.sk > 128) {
        res.status = GENIOS_EUNSUPPORTED;
        res.err = "lockstep batch: K and the sketch rank must be in 1..128";
        return res;
    }
    Ctx c{};
    c.m = m;
    c.n = n;
    c.K = K;
    c.Kp = (int)rup(K, 8);
    c.sk = in.sk;
    c.ldn = rup(n, 32);
    c.rpad_m = rup(m, 128);
    c.kpad_n = rup(n, 64);
    c.rpad_n = rup(n, 128);
    c.kpad_m = rup(m, 64);
    c.s1 = tc_splits_for(c.rpad_m / 128, c.kpad_n / 64);
    c.s2 = tc_splits_for(c.rpad_n / 128, c.kpad_m / 64);
    c.wait = in.wait_limit;
    c.s = in.stream;
    Buf buf;
    const size_t ab = (size_t)c.rpad_m * c.kpad_n * 2, atb = (size_t)c.rpad_n * c.kpad_m * 2;
    const size_t nk = (size_t)c.ldn * K * 4;
    float *X, *Z, *U, *G, *R, *Dl, *P, *Q, *Y, *Cw;
    double *part, *part_w;
    BState* BS;
    const int nb = (int)((n + BK_RB - 1) / BK_RB);
    // rows per block of the U^T R / U C kernels: U rows and R columns staged in ~200 KB of smem
    const int urb = (int)std::max<int64_t>(32, std::min<int64_t>(512, ((200 * 1024) / (4 * (std::max(1, in.sk) + K))) / 32 * 32));
    const int nbu = (int)((n + urb - 1) / urb);
    cudaError_t e = cudaSuccess;
#define BGET(p, b) if (e == cudaSuccess) e = buf.get((void**)&(p), (b))
    BGET(c.Ah_rows, ab); BGET(c.Al_rows, ab); BGET(c.Ah_cols, atb); BGET(c.Al_cols, atb);
    BGET(c.Bx, (size_t)2 * c.Kp * c.kpad_n * 2); BGET(c.Bw, (size_t)2 * c.Kp * c.kpad_m * 2);
    BGET(c.part1a, (size_t)c.s1 * c.rpad_m * 2 * c.Kp * 4); BGET(c.part1b, (size_t)c.s1 * c.rpad_m * 2 * c.Kp * 4);
    BGET(c.part2a, (size_t)c.s2 * c.rpad_n * 2 * c.Kp * 4); BGET(c.part2b, (size_t)c.s2 * c.rpad_n * 2 * c.Kp * 4);
    BGET(c.err, 256);
    BGET(X, nk); BGET(Z, nk); BGET(U, nk); BGET(G, nk); BGET(R, nk); BGET(Dl, nk); BGET(P, nk); BGET(Q, nk); BGET(Y, nk);
    BGET(Cw, (size_t)K * std::max(1, c.sk) * 4);
    BGET(part, (size_t)nb * K * BK_NV * 8);
    BGET(part_w, (size_t)nbu * K * std::max(1, c.sk) * 8);
    BGET(BS, (size_t)K * sizeof(BState));
#undef BGET
    if (e != cudaSuccess) {
        res.status = GENIOS_ENOMEM;
        res.err = std::string("lockstep batch: ") + cudaGetErrorString(e);
        return res;
    }
    cudaStream_t s = c.s;
    // operands: bf16 hi / lo of A and A^T
    TcPlan tp = tc_plan(m, n, std::max(1, std::min(c.sk, 128)));
    TcWork hw{};
    hw.A_rows = c.Ah_rows;
    hw.A_cols = c.Ah_cols;
    TcWork lw{};
    lw.A_rows = c.Al_rows;
    lw.A_cols = c.Al_cols;
    e = tc_pack_a(tp, hw, P_FP32, in.A, in.lda, nullptr, s);
    if (e == cudaSuccess) e = batch_pack_lo(tp, lw, in.A, in.lda, s);
    cudaMemsetAsync(X, 0, nk, s);
    cudaMemsetAsync(Z, 0, nk, s);
    cudaMemsetAsync(U, 0, nk, s);
    cudaMemsetAsync(c.err, 0, 256, s);
    std::vector<BState> h(K);
    std::vector<double> rho(K, in.rho0);
    std::vector<int> n_rho(K, 0), iters(K, 0), conv(K, 0);
    std::vector<KktSchedule> kkt(K, KktSchedule(in.kkt_every, -1000000));
    std::vector<double> last_rp(K, 0.0), last_rd(K, 0.0);
    for (int k = 0; k < K; ++k) {
        BState& b = h[k];
        b = BState{};
        b.rho = in.rho0;
        b.lam1 = in.lam1[k];
        b.lam2 = in.lam2[k];
        b.nu = in.rho0 + in.lam2[k];
        b.u_scale = 1.0;
        b.active = 1;
        b.cg_max = in.max_cg;
    }
    auto push = [&]() { return cudaMemcpyAsync(BS, h.data(), K * sizeof(BState), cudaMemcpyHostToDevice, s); };
    auto pull = [&]() {
        cudaError_t x = cudaMemcpyAsync(h.data(), BS, K * sizeof(BState), cudaMemcpyDeviceToHost, s);
        if (x == cudaSuccess) x = cudaStreamSynchronize(s);
        return x;
    };
    if (e == cudaSuccess) e = push();
    const dim3 gcol((unsigned)nb, (unsigned)K);
    const size_t ut_smem = (size_t)(urb * c.sk + K * urb) * 4;
    const size_t uc_smem = (size_t)(urb * c.sk + K * c.sk) * 4;
    if (e == cudaSuccess && c.sk > 0) {
        cudaFuncSetAttribute(bk_ut_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ut_smem + 1024);
        cudaFuncSetAttribute(bk_uc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)uc_smem + 1024);
    }
    const double sqn = std::sqrt((double)n);
    int64_t launches = 0, cg_total = 0;
    int k_iter = 0;
    auto precond = [&](int start) -> cudaError_t {
        // Zc = P^{-1} R (Eq. (10)) into P (start: P = Zc; otherwise P = Zc + beta P)
        if (c.sk == 0) return cudaErrorInvalidValue;
        bk_ut_kernel<<<nbu, BK_T, ut_smem, s>>>(n, c.ldn, K, c.sk, urb, in.U, R, part_w);
        bk_w_kernel<<<K, 128, 0, s>>>(start, nbu, K, c.sk, part_w, in.lam, BS, Cw);
        bk_uc_kernel<<<nbu, BK_T, uc_smem, s>>>(n, c.ldn, K, c.sk, urb, in.U, R, Cw, BS, start, P);
        launches += 3;
        return cudaGetLastError();
    };
    for (k_iter = 1; e == cudaSuccess && k_iter <= in.max_iter; ++k_iter) {
        // gradient at x for every active problem (accurate products)
        e = ata(c, X, Y, true);
        if (e != cudaSuccess) break;
        bk_grad_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, Y, in.g0, X, U, BS, G, part);
        bk_reduce_kernel<<<K, 256, 0, s>>>(RED_GRAD, nb, part, BS);
        launches += 10;
        if ((e = pull()) != cudaSuccess) break;
        // residuals (Eqs. (11)-(12)), stop tests, penalty updates, CG tolerances: host logic
        bool any = false, need_kkt = false;
        std::vector<int> check(K, 0);
        for (int k = 0; k < K; ++k) {
            BState& b = h[k];
            if (!b.active) continue;
            if (k_iter > 1) {
                const double rp = std::sqrt(b.rp2), rd = std::sqrt(b.rd2);
                last_rp[k] = rp;
                last_rd[k] = rd;
                const bool resid_ok = rp <= sqn * in.eps_abs + in.eps_rel * std::max(std::sqrt(b.x2), std::sqrt(b.z2)) &&
                                      rd <= sqn * in.eps_abs + in.eps_rel * std::sqrt(b.rhou2);
                if (kkt[k].due(k_iter, resid_ok)) {
                    check[k] = 1;
                    need_kkt = true;
                }
            }
        }
        if (need_kkt) {
            e = ata(c, Z, Y, true);
            if (e != cudaSuccess) break;
            bk_kkt_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, Y, in.g0, Z, BS, part);
            bk_reduce_kernel<<<K, 256, 0, s>>>(RED_KKT, nb, part, BS);
            launches += 10;
            if ((e = pull()) != cudaSuccess) break;
            for (int k = 0; k < K; ++k) {
                if (!check[k]) continue;
                BState& b = h[k];
                const double rk = std::sqrt(b.kd2) / std::max(std::max(std::sqrt(b.kg2), b.lam1), 1e-30);
                kkt[k].record(k_iter, rk, in.eps_kkt);
                info[k].rel_kkt = rk;
                if (rk <= in.eps_kkt) {
                    b.active = 0;
                    conv[k] = 1;
                    iters[k] = k_iter - 1;
                }
            }
        }
        for (int k = 0; k < K; ++k) {
            BState& b = h[k];
            if (!b.active) continue;
            any = true;
            b.u_scale = 1.0;
            if (k_iter > 1 && in.rho_every > 0 && (k_iter - 1) % in.rho_every == 0 && n_rho[k] < in.rho_max &&
                k_iter <= in.rho_until) {
                double nr = b.rho;
                if (last_rp[k] > in.rho_mu * last_rd[k]) nr = b.rho * in.rho_tau;
                else if (last_rd[k] > in.rho_mu * last_rp[k]) nr = b.rho / in.rho_tau;
                if (nr != b.rho) {
                    b.u_scale = b.rho / nr;
                    b.rho = nr;
                    n_rho[k]++;
                }
            }
            b.nu = b.rho + b.lam2;
            double tol = k_iter <= 1 ? in.cg_first
                                     : std::min(std::sqrt(last_rp[k] * last_rd[k]), 1.0) / std::pow((double)k_iter, in.gamma);
            b.tol = std::max(tol, in.cg_floor);
            iters[k] = k_iter;
        }
        if (!any) break;
        if ((e = push()) != cudaSuccess) break;
        // x-subproblem for every active problem: batched PCG on (A^T A + nu_k I) delta = r
        bk_rhs_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, G, X, Z, U, BS, R, Dl, part);
        bk_reduce_kernel<<<K, 256, 0, s>>>(RED_RHS, nb, part, BS);
        launches += 2;
        e = precond(1);
        if (e != cudaSuccess) break;
        for (int it = 0; it < in.max_cg + 1; ++it) {
            if ((e = pull()) != cudaSuccess) break;
            bool cg_any = false;
            for (int k = 0; k < K; ++k) cg_any = cg_any || h[k].cg_active;
            if (!cg_any) break;
            e = ata(c, P, Q, false);   // Q = A^T A P (bf16 A)
            if (e != cudaSuccess) break;
            bk_q_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, Q, P, BS, Q, part);
            bk_reduce_kernel<<<K, 256, 0, s>>>(RED_Q, nb, part, BS);
            bk_upd_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, P, Q, BS, R, Dl, part);
            bk_reduce_kernel<<<K, 256, 0, s>>>(RED_UPD, nb, part, BS);
            launches += 9;
            e = precond(0);
            if (e != cudaSuccess) break;
            cg_total += 1;
        }
        if (e != cudaSuccess) break;
        bk_zu_kernel<<<gcol, BK_T, 0, s>>>(n, c.ldn, Dl, X, Z, U, in.alpha, BS, part);
        bk_reduce_kernel<<<K, 256, 0, s>>>(RED_ZU, nb, part, BS);
        launches += 2;
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = pull();
    if (e == cudaSuccess) {
        // z of every problem, back to back
        for (int k = 0; k < K; ++k) {
            e = cudaMemcpyAsync(static_cast<float*>(in.z_out) + (size_t)k * n, Z + (size_t)k * c.ldn, (size_t)n * 4,
                                cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        res.status = GENIOS_ECUDA;
        res.err = std::string("lockstep batch: ") + cudaGetErrorString(e);
        return res;
    }
    if (herr) {
        res.status = GENIOS_ETIMEOUT;
        res.err = "lockstep batch: a bounded wait in the tensor-core products ran out";
        return res;
    }
    for (int k = 0; k < K; ++k) {
        genios_info& f = info[k];
        f.status = conv[k] ? GENIOS_OK : GENIOS_EMAXITER;
        f.iters = conv[k] ? iters[k] : in.max_iter;
        f.rho = h[k].rho;
        f.rho_updates = n_rho[k];
        f.lambda1 = in.lam1[k];
        f.lambda2 = in.lam2[k];
        f.r_p = std::sqrt(h[k].rp2);
        f.r_d = std::sqrt(h[k].rd2);
        f.nnz = (int)h[k].nnz;
        if (!conv[k]) res.status = GENIOS_EMAXITER;
    }
    res.iterations = k_iter - 1;
    res.cg_iterations = cg_total;
    res.launches = launches;
    return res;
}

}  // namespace genios
