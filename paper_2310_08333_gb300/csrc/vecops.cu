// n-vector and m-vector kernels of the ADMM iteration (sm_103a).
//
// All reductions are deterministic: per-block sums in a fixed shape, then the last block to
// finish adds the block partials in block order (grid_sum).  Scalars that later kernels need
// stay on the device in DevState.  Kernels of the CG loop return at once when
// DevState::cg_done is set, so a loop body can be replayed (CUDA graph) after convergence.
#include "common.cuh"
#include "internal.h"
#include "genios.h"
#include "devloop.cuh"

namespace genios {

constexpr int VT_THREADS = 256;

static inline int nblocks(int64_t n, int per) { return (int)((n + per - 1) / per); }

// Sum of column j of the G x ldp partial matrix, computed by the 8 warps of a 256-thread block
// for 32 consecutive columns.  Returns the column sum in warp 0 lanes (others: 0).
template <typename VT, typename AccT>
GENIOS_DEV AccT column_sum(const VT* P, int G, int64_t ldp, int64_t j, int64_t n, AccT* sh) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    AccT acc = AccT(0);
    if (j < n)
        for (int b = ty; b < G; b += 8) acc += (AccT)P[(int64_t)b * ldp + j];
    sh[ty * 33 + tx] = acc;
    __syncthreads();
    AccT out = AccT(0);
    if (ty == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) out += sh[k * 33 + tx];
    }
    __syncthreads();
    return out;
}

// ------------------------------------------------------------------------------------------
template <typename VT>
__global__ void hv_finish_kernel(const VT* P, int G, int64_t ldp, int64_t n, double nu,
                                 const VT* v, VT* y) {
    __shared__ VT sh[8 * 33];
    const int64_t j = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    VT sum = column_sum<VT, VT>(P, G, ldp, j, n, sh);
    if ((threadIdx.x >> 5) == 0 && j < n) y[j] = sum + (VT)nu * v[j];
}

// U^T r over the block's UTR_ROWS rows (r staged in shared memory) plus the block sum of r^2.
// Threads: c = t % 128 is a column of U, g = t / 128 one of two row groups; products and the
// per-thread sums run in the value type, block partials in float64.  The last block adds the
// partials of all blocks in a fixed order (two threads per column, four independent
// accumulators each) into w_out and returns true with rr_out.  Requires s <= 128, blockDim 256.
constexpr int UTR_ROWS = 64;

template <typename VT>
GENIOS_DEV bool ut_r_and_norm(const VT* U, int sk, const VT* rsh, int64_t j0, int64_t n,
                              double rr_thread, double* part, unsigned* counter,
                              double* w_out, double& rr_out, long long* dbg) {
    const int t = threadIdx.x;
    const int c = t & 127, g = t >> 7;
    __shared__ double wsh[256];
    __shared__ unsigned s_last;
    __shared__ double s_rr;
    VT acc = VT(0);
    if (c < sk) {
        const int rows = (int)min((int64_t)UTR_ROWS, n - j0);
        for (int jj = g; jj < rows; jj += 2)
            if (GCHK(dbg, (j0 + jj) * sk + c, n * (long long)sk))
                acc = fma(U[(j0 + jj) * sk + c], rsh[jj], acc);
    }
    wsh[t] = (double)acc;
    double v[1] = {rr_thread};
    block_sum<1>(v);  // its barriers also publish wsh
    const int stride = sk + 1;
    if (t < sk && GCHK(dbg, (long long)blockIdx.x * stride + t, 262144))
        part[(size_t)blockIdx.x * stride + t] = wsh[t] + wsh[t + 128];
    if (t == 0 && GCHK(dbg, (long long)blockIdx.x * stride + sk, 262144))
        part[(size_t)blockIdx.x * stride + sk] = v[0];
    __threadfence();
    __syncthreads();
    if (t == 0) {
        unsigned k = atomicAdd(counter, 1u);
        s_last = (k == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int nb = gridDim.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (c < sk) {
        int b = g;
        for (; b + 6 < nb; b += 8) {
            a0 += __ldcg(part + (size_t)b * stride + c);
            a1 += __ldcg(part + (size_t)(b + 2) * stride + c);
            a2 += __ldcg(part + (size_t)(b + 4) * stride + c);
            a3 += __ldcg(part + (size_t)(b + 6) * stride + c);
        }
        for (; b < nb; b += 2) a0 += __ldcg(part + (size_t)b * stride + c);
    }
    __syncthreads();
    wsh[t] = (a0 + a1) + (a2 + a3);
    if (t < 32) {  // r^2 slot
        double r2 = 0.0;
        for (int b = t; b < nb; b += 32) r2 += __ldcg(part + (size_t)b * stride + sk);
        r2 = warp_sum(r2);
        if (t == 0) s_rr = r2;
    }
    __syncthreads();
    if (t < sk && GCHK(dbg, t, 256)) w_out[t] = wsh[t] + wsh[t + 128];
    rr_out = s_rr;
    if (t == 0) *counter = 0u;
    return true;
}

template <typename VT>
__global__ void cg_precond_kernel(int64_t n, const VT* U, int sk, const double* lam, const VT* r,
                                  VT* zc, DevState* S, Scratch sc) {
    if (S->cg_done) return;
    __shared__ VT coefw[256];
    const double nu = S->nu;
    const double ls = lam[sk - 1];
    for (int c = threadIdx.x; c < sk; c += blockDim.x)
        if (GCHK(sc.dbg, c, 256)) coefw[c] = (VT)(((ls + nu) / (lam[c] + nu) - 1.0) * S->w[c]);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    double rz = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * nw + wid; j < n; j += (int64_t)gridDim.x * nw) {
        VT acc = VT(0);
        for (int c = lane; c < sk; c += 32)
            if (GCHK(sc.dbg, j * sk + c, n * (long long)sk)) acc = fma(U[j * sk + c], coefw[c], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const VT rj = r[j];
            const VT zj = rj + acc;
            zc[j] = zj;
            rz += (double)rj * (double)zj;
        }
    }
    double v[1] = {rz}, out[1];
    if (grid_sum<1>(v, sc.part, sc.counter, out)) {
        if (threadIdx.x == 0) {
            if (S->cg_first) {
                S->beta = 0.0;
                S->cg_first = 0;
            } else {
                S->beta = S->rz > 0.0 ? out[0] / S->rz : 0.0;
            }
            S->rz = out[0];
        }
    }
}

template <typename VT>
__global__ void rhs_init_kernel(int64_t n, const VT* g, const VT* x, const VT* z, VT* u, double rho,
                                double u_scale, double nu, double tol, int cg_max, VT* r, VT* delta,
                                VT* p, VT* zc, const VT* U, int sk, DevState* S, Scratch sc) {
    __shared__ VT rsh[UTR_ROWS];
    const int64_t j0 = (int64_t)blockIdx.x * UTR_ROWS;
    const int64_t j = j0 + threadIdx.x;
    double rr = 0.0;
    if (threadIdx.x < UTR_ROWS) {
        VT rj = VT(0);
        if (j < n) {
            const VT uj = u[j] * (VT)u_scale;
            u[j] = uj;
            rj = -(g[j] + (VT)rho * (x[j] - z[j] + uj));
            r[j] = rj;
            delta[j] = VT(0);
            p[j] = VT(0);
            if (sk == 0) zc[j] = rj;
            rr = (double)rj * (double)rj;
        }
        rsh[threadIdx.x] = rj;
    }
    __syncthreads();
    double rr_tot;
    if (ut_r_and_norm<VT>(U, sk, rsh, j0, n, rr, sc.part, sc.counter, S->w, rr_tot, sc.dbg)) {
        if (threadIdx.x == 0) {
            S->rhs2 = rr_tot;
            S->rr = rr_tot;
            S->nu = nu;
            S->tol = tol;
            S->cg_it = 0;
            S->cg_max = cg_max;
            S->cg_done = rr_tot > 0.0 ? 0 : 1;
            S->cg_first = 1;
            S->cg_guard = 0;
            S->hv_t0 = ~0ull;
            S->hv_t1 = 0ull;
            S->beta = 0.0;
            if (sk == 0) {
                S->rz = rr_tot;
                S->cg_first = 0;
            }
        }
    }
}

template <typename VT>
__global__ void grad_finish_kernel(const VT* P, int G, int64_t ldp, const double* loss_part,
                                   int64_t n, const VT* x, const VT* u, double mu, double rho,
                                   double lam1, VT* g, DevState* S, Scratch sc, DevLoop* loop,
                                   cudaGraphConditionalHandle kkt_cond, cudaGraphConditionalHandle loop_cond,
                                   int use_cond) {
    double kpow_next = 0.0;   // k^gamma for phase b (phase a makes this iteration k + 1), read early
    if (loop != nullptr) {   // device-side loop: nothing to do once it halted (uniform across the grid)
        if (loop->halt) return;
        rho = loop->rho;
        mu = loop->lam2;
        lam1 = loop->lam1;
        if (threadIdx.x == 0) kpow_next = loop_kpow(loop, loop->k + 1);
    }
    __shared__ double sh[8 * 33];
    const int64_t j = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    double sum = column_sum<VT, double>(P, G, ldp, j, n, sh);
    double v[6] = {0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    if ((threadIdx.x >> 5) == 0 && j < n) {
        // explicit roundings: the fused finish of the persistent CG kernel forms the same values
        const double xj = (double)x[j];
        const double gj = fma(mu, xj, sum);
        g[j] = (VT)gj;
        const double rhou = __dmul_rn(rho, (double)u[j]);
        const double rd = __dadd_rn(gj, rhou);
        const double atw = fabs(sum);
        const double ex = fmax(atw - lam1, 0.0);
        v[0] = rd * rd;
        v[1] = rhou * rhou;
        v[2] = gj * gj;
        v[3] = ex * ex;
        v[4] = fabs(xj);
        v[5] = xj * xj;
        mx[0] = atw;
    }
    double out[6], outm[1];
    if (grid_sum_max<6, 1>(v, mx, sc.part, sc.counter, out, outm)) {
        double ls[1] = {0.0};
        for (int b = threadIdx.x; b < G; b += blockDim.x) ls[0] += loss_part[b];
        block_sum<1>(ls);
        auto fill = [&](DevState* T) {
            T->loss_sum = ls[0];
            T->rd2 = out[0];
            T->rhou2 = out[1];
            T->g2 = out[2];
            T->excess2 = out[3];
            T->gx1 = out[4];
            T->gx2 = out[5];
            T->atw_inf = outm[0];
        };
        if (loop == nullptr) {
            if (threadIdx.x == 0) fill(S);
            return;
        }
        __shared__ unsigned long long head[kStateHeadBytes / 8];
        loop_decide_shared(
            S, head, threadIdx.x, blockDim.x, [] { __syncthreads(); },
            [&](DevState* Ss) {
                fill(Ss);
                fill(S);
            },
            [&](DevLoop* Lc, DevState* Ss) {
                loop_phase_a(Lc, Ss);
                if (Lc->skip_kkt) loop_phase_b(Lc, Ss, kpow_next);
                if (use_cond) {
                    cudaGraphSetConditional(kkt_cond, Lc->skip_kkt ? 0u : 1u);
                    if (Lc->skip_kkt) cudaGraphSetConditional(loop_cond, Lc->cont ? 1u : 0u);
                }
            });
    }
}

template <typename VT>
__global__ void kkt_finish_kernel(const VT* P, int G, int64_t ldp, int64_t n, const VT* z,
                                  double mu, double lam1, DevState* S, Scratch sc, int box, double lo,
                                  double hi, DevLoop* loop, cudaGraphConditionalHandle loop_cond,
                                  int use_cond) {
    double kpow_k = 0.0;   // k^gamma for phase b, read early
    if (loop != nullptr) {
        if (loop->skip_kkt) return;   // no check due (uniform across the grid)
        mu = loop->lam2;
        lam1 = loop->lam1;
        if (threadIdx.x == 0) kpow_k = loop_kpow(loop, loop->k);
    }
    __shared__ double sh[8 * 33];
    const int64_t j = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    double sum = column_sum<VT, double>(P, G, ldp, j, n, sh);
    double v[2] = {0, 0};
    double mx[1] = {0.0};
    if ((threadIdx.x >> 5) == 0 && j < n) {
        const double zj = (double)z[j];
        const double gj = sum + mu * zj;
        double d;
        if (box) {   // distance of 0 from g + N(z), N the normal cone of the box at z
            if (zj <= lo) d = fmax(-gj, 0.0);
            else if (zj >= hi) d = fmax(gj, 0.0);
            else d = fabs(gj);
        } else if (zj > 0.0) d = fabs(gj + lam1);
        else if (zj < 0.0) d = fabs(gj - lam1);
        else d = fmax(fabs(gj) - lam1, 0.0);
        v[0] = d * d;
        v[1] = gj * gj;
        mx[0] = d;
    }
    // the block's butterfly sums (warp 0 holds its 32 columns), then in the last block to finish
    // one warp per total over the blocks (warp_total)
    __shared__ unsigned s_last;
    __shared__ double tot[3];
    if ((threadIdx.x >> 5) == 0) {
        v[0] = warp_sum(v[0]);
        v[1] = warp_sum(v[1]);
        mx[0] = warp_max(mx[0]);
        if (threadIdx.x == 0) {
            sc.part[(size_t)blockIdx.x * 4 + 0] = v[0];
            sc.part[(size_t)blockIdx.x * 4 + 1] = v[1];
            sc.part[(size_t)blockIdx.x * 4 + 2] = mx[0];
            __threadfence();
            s_last = atomicAdd(sc.counter, 1u) == gridDim.x - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    {
        const int wid = threadIdx.x >> 5;
        if (wid < 3) {
            const double t = warp_total(sc.part + wid, (int)gridDim.x, 4, wid == 2);
            if ((threadIdx.x & 31) == 0) tot[wid] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
    {
        auto fill = [&](DevState* T) {
            T->kd2 = tot[0];
            T->kg2 = tot[1];
            T->kdmax = tot[2];
        };
        if (loop == nullptr) {
            if (threadIdx.x == 0) fill(S);
            return;
        }
        __shared__ unsigned long long head[kStateHeadBytes / 8];
        loop_decide_shared(
            S, head, threadIdx.x, blockDim.x, [] { __syncthreads(); },
            [&](DevState* Ss) {
                fill(Ss);
                fill(S);
            },
            [&](DevLoop* Lc, DevState* Ss) {
                loop_phase_b(Lc, Ss, kpow_k);
                if (use_cond) cudaGraphSetConditional(loop_cond, Lc->cont ? 1u : 0u);
            });
    }
}

template <typename VT>
__global__ void gap_kernel(int loss, int64_t m, const VT* W, const VT* b, double mu, double lam1,
                           DevState* S, Scratch sc) {
    const double scale = (mu == 0.0 && S->atw_inf > lam1) ? lam1 / S->atw_inf : 1.0;
    double v[2] = {0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double nu = scale * (double)W[i];
        v[0] += loss_conj(loss, nu);
        v[1] += (double)b[i] * nu;
    }
    double out[2];
    if (grid_sum<2>(v, sc.part, sc.counter, out)) {
        if (threadIdx.x == 0) {
            S->conj_sum = out[0];
            S->btnu = out[1];
            S->gap_scale = scale;
        }
    }
}

template <typename VT>
__global__ void zu_kernel(int64_t n, VT* x, const VT* delta, VT* z, VT* u, double rho, double lam1,
                          double alpha, DevState* S, double* norms_out, Scratch sc, int box, double lo,
                          double hi) {
    const double kappa = lam1 / rho;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        VT xj = x[j];
        if (delta != nullptr) {
            xj += delta[j];
            x[j] = xj;
        }
        const VT zj = z[j];
        const VT xh = (VT)alpha * xj + (VT)(1.0 - alpha) * zj;
        const VT vv = xh + u[j];
        VT zn;
        if (box) zn = vv < (VT)lo ? (VT)lo : vv > (VT)hi ? (VT)hi : vv;   // projection onto the box
        else if (vv > (VT)kappa) zn = vv - (VT)kappa;
        else if (vv < -(VT)kappa) zn = vv + (VT)kappa;
        else zn = VT(0);
        const VT un = u[j] + xh - zn;
        z[j] = zn;
        u[j] = un;
        const double dxz = (double)xj - (double)zn;
        v[0] += dxz * dxz;
        v[1] += (double)xj * (double)xj;
        v[2] += (double)zn * (double)zn;
        v[3] += (double)un * (double)un;
        v[4] += fabs((double)zn);
        v[5] += zn != VT(0) ? 1.0 : 0.0;
    }
    double out[6];
    if (grid_sum<6>(v, sc.part, sc.counter, out)) {
        if (threadIdx.x == 0) {
            if (S) {
                S->rp2 = out[0];
                S->x2 = out[1];
                S->z2 = out[2];
                S->u2 = out[3];
                S->z1 = out[4];
                S->nnz = out[5];
            }
            if (norms_out)
                for (int k = 0; k < 6; ++k) norms_out[k] = out[k];
        }
    }
}

// ------------------------------------------------------------------------------------------
template <typename S, typename D>
__global__ void convert_kernel(int64_t rows, int64_t cols, const S* src, int64_t lds, D* dst,
                               int64_t ldd) {
    const int64_t total = rows * ldd;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldd, j = e % ldd;
        dst[e] = j < cols ? (D)src[i * lds + j] : D(0);
    }
}

// ------------------------------------------------------------------------------------------
// implicit gradient (adjoint of the optimality conditions on the support)
// ------------------------------------------------------------------------------------------
// r = g restricted to the support of z (z_j != 0), from a float64 gradient
template <typename VT>
__global__ void adj_rhs_kernel(int64_t n, const double* g, const VT* z, VT* r) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        r[j] = z[j] != VT(0) ? (VT)g[j] : VT(0);
}

// out[0] = -sum_j q_j sign(z_j)   (one block, fixed order)
template <typename VT>
__global__ void adj_lambda_kernel(int64_t n, const VT* q, const VT* z, double* out) {
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const VT zj = z[j];
        if (zj != VT(0)) acc -= (double)q[j] * (zj > VT(0) ? 1.0 : -1.0);
    }
    double v[1] = {acc};
    block_sum<1>(v);
    if (threadIdx.x == 0) out[0] = v[0];
}

// dL/db_i = D_i t_i with t = A q (float64 output)
template <typename VT>
__global__ void adj_db_kernel(int64_t m, const VT* t, const VT* D, double* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)D[i] * (double)t[i];
}

// dL/dA = -(l'(t_z) q^T + (D A q) z^T), m x n float64 row-major with row stride ld
template <typename VT>
__global__ void adj_da_kernel(int64_t m, int64_t n, const VT* l1, const VT* q, const VT* D, const VT* t,
                              const VT* z, double* out, int64_t ld) {
    const int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        out[i * ld + j] = -((double)l1[i] * (double)q[j] + (double)D[i] * (double)t[i] * (double)z[j]);
    }
}

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
static int grid_for(int64_t n, int per, int cap = 4096) {
    int g = nblocks(n, per);
    return g < 1 ? 1 : (g > cap ? cap : g);
}

#define DISPATCH_VT(dbl, KERNEL, GRID, BLOCK, ST, ...)                                     \
    do {                                                                                  \
        if (dbl) KERNEL<double><<<GRID, BLOCK, 0, ST>>>(__VA_ARGS__);                     \
        else KERNEL<float><<<GRID, BLOCK, 0, ST>>>(__VA_ARGS__);                          \
    } while (0)

template <typename VT> static VT* C(void* p) { return static_cast<VT*>(p); }
template <typename VT> static const VT* CC(const void* p) { return static_cast<const VT*>(p); }

cudaError_t hv_finish(bool dbl, const void* P, int G, int64_t ldp, int64_t n, double nu,
                      const void* v, void* y, cudaStream_t s) {
    const int grid = nblocks(n, 32);
    if (dbl) hv_finish_kernel<double><<<grid, VT_THREADS, 0, s>>>(CC<double>(P), G, ldp, n, nu, CC<double>(v), C<double>(y));
    else hv_finish_kernel<float><<<grid, VT_THREADS, 0, s>>>(CC<float>(P), G, ldp, n, nu, CC<float>(v), C<float>(y));
    return cudaGetLastError();
}

// per-block partials of U^T r must fit the scratch partial buffer
static bool utr_fits(int64_t n, int sk) {
    return sk <= 128 && (int64_t)nblocks(n, UTR_ROWS) * (sk + 1) <= 262144;
}

cudaError_t cg_precond(bool dbl, int64_t n, const void* U, int sk, const double* lam, const void* r,
                       void* zc, DevState* S, Scratch sc, cudaStream_t s) {
    const int grid = grid_for(n, 8, 608);
    if (dbl) cg_precond_kernel<double><<<grid, VT_THREADS, 0, s>>>(n, CC<double>(U), sk, lam, CC<double>(r), C<double>(zc), S, sc);
    else cg_precond_kernel<float><<<grid, VT_THREADS, 0, s>>>(n, CC<float>(U), sk, lam, CC<float>(r), C<float>(zc), S, sc);
    return cudaGetLastError();
}

cudaError_t rhs_init(bool dbl, int64_t n, const void* g, const void* x, const void* z, void* u,
                     double rho, double u_scale, double nu, double tol, int cg_max, void* r,
                     void* delta, void* p, void* zc, const void* U, int sk, DevState* S,
                     Scratch sc, cudaStream_t s) {
    if (!utr_fits(n, sk)) return cudaErrorInvalidValue;
    const int grid = nblocks(n, UTR_ROWS);
    if (dbl) rhs_init_kernel<double><<<grid, VT_THREADS, 0, s>>>(n, CC<double>(g), CC<double>(x), CC<double>(z), C<double>(u), rho, u_scale, nu, tol, cg_max, C<double>(r), C<double>(delta), C<double>(p), C<double>(zc), CC<double>(U), sk, S, sc);
    else rhs_init_kernel<float><<<grid, VT_THREADS, 0, s>>>(n, CC<float>(g), CC<float>(x), CC<float>(z), C<float>(u), rho, u_scale, nu, tol, cg_max, C<float>(r), C<float>(delta), C<float>(p), C<float>(zc), CC<float>(U), sk, S, sc);
    return cudaGetLastError();
}

cudaError_t grad_finish(bool dbl, const void* P, int G, int64_t ldp, const double* loss_part,
                        int64_t n, const void* x, const void* u, double mu, double rho,
                        double lam1, void* g, DevState* S, Scratch sc, cudaStream_t s, DevLoop* loop,
                        unsigned long long kkt_cond, unsigned long long loop_cond, int use_cond) {
    const int grid = nblocks(n, 32);
    if (dbl) grad_finish_kernel<double><<<grid, VT_THREADS, 0, s>>>(CC<double>(P), G, ldp, loss_part, n, CC<double>(x), CC<double>(u), mu, rho, lam1, C<double>(g), S, sc, loop, (cudaGraphConditionalHandle)kkt_cond, (cudaGraphConditionalHandle)loop_cond, use_cond);
    else grad_finish_kernel<float><<<grid, VT_THREADS, 0, s>>>(CC<float>(P), G, ldp, loss_part, n, CC<float>(x), CC<float>(u), mu, rho, lam1, C<float>(g), S, sc, loop, (cudaGraphConditionalHandle)kkt_cond, (cudaGraphConditionalHandle)loop_cond, use_cond);
    return cudaGetLastError();
}

cudaError_t kkt_finish(bool dbl, const void* P, int G, int64_t ldp, int64_t n, const void* z,
                       double mu, double lam1, DevState* S, Scratch sc, cudaStream_t s, int box, double lo,
                       double hi, DevLoop* loop, unsigned long long loop_cond, int use_cond) {
    const int grid = nblocks(n, 32);
    if (dbl) kkt_finish_kernel<double><<<grid, VT_THREADS, 0, s>>>(CC<double>(P), G, ldp, n, CC<double>(z), mu, lam1, S, sc, box, lo, hi, loop, (cudaGraphConditionalHandle)loop_cond, use_cond);
    else kkt_finish_kernel<float><<<grid, VT_THREADS, 0, s>>>(CC<float>(P), G, ldp, n, CC<float>(z), mu, lam1, S, sc, box, lo, hi, loop, (cudaGraphConditionalHandle)loop_cond, use_cond);
    return cudaGetLastError();
}



cudaError_t gap_pieces(bool dbl, int loss, int64_t m, const void* W, const void* b, double mu,
                       double lam1, DevState* S, Scratch sc, cudaStream_t s) {
    const int grid = grid_for(m, VT_THREADS, 512);
    if (dbl) gap_kernel<double><<<grid, VT_THREADS, 0, s>>>(loss, m, CC<double>(W), CC<double>(b), mu, lam1, S, sc);
    else gap_kernel<float><<<grid, VT_THREADS, 0, s>>>(loss, m, CC<float>(W), CC<float>(b), mu, lam1, S, sc);
    return cudaGetLastError();
}

cudaError_t zu_update(bool dbl, int64_t n, void* x, const void* delta, void* z, void* u,
                      double rho, double lam1, double alpha, DevState* S, double* norms_out,
                      Scratch sc, cudaStream_t s, int box, double lo, double hi) {
    const int grid = grid_for(n, VT_THREADS, 512);
    if (dbl) zu_kernel<double><<<grid, VT_THREADS, 0, s>>>(n, C<double>(x), CC<double>(delta), C<double>(z), C<double>(u), rho, lam1, alpha, S, norms_out, sc, box, lo, hi);
    else zu_kernel<float><<<grid, VT_THREADS, 0, s>>>(n, C<float>(x), CC<float>(delta), C<float>(z), C<float>(u), rho, lam1, alpha, S, norms_out, sc, box, lo, hi);
    return cudaGetLastError();
}

cudaError_t convert_copy(int src_dt, int dst_dt, int64_t rows, int64_t cols, const void* src,
                         int64_t lds, void* dst, int64_t ldd, cudaStream_t s) {
    const int grid = grid_for(rows * ldd, VT_THREADS, 152 * 16);
    // dtype codes: 0 f64, 1 f32
    if (src_dt == 0 && dst_dt == 0) convert_kernel<double, double><<<grid, VT_THREADS, 0, s>>>(rows, cols, CC<double>(src), lds, C<double>(dst), ldd);
    else if (src_dt == 0 && dst_dt == 1) convert_kernel<double, float><<<grid, VT_THREADS, 0, s>>>(rows, cols, CC<double>(src), lds, C<float>(dst), ldd);
    else if (src_dt == 1 && dst_dt == 0) convert_kernel<float, double><<<grid, VT_THREADS, 0, s>>>(rows, cols, CC<float>(src), lds, C<double>(dst), ldd);
    else if (src_dt == 1 && dst_dt == 1) convert_kernel<float, float><<<grid, VT_THREADS, 0, s>>>(rows, cols, CC<float>(src), lds, C<float>(dst), ldd);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t fill_zero(void* p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

}  // namespace genios

namespace genios {
cudaError_t adj_rhs(bool dbl, int64_t n, const double* g, const void* z, void* r, cudaStream_t s) {
    const int grid = grid_for(n, VT_THREADS, 1024);
    if (dbl) adj_rhs_kernel<double><<<grid, VT_THREADS, 0, s>>>(n, g, CC<double>(z), C<double>(r));
    else adj_rhs_kernel<float><<<grid, VT_THREADS, 0, s>>>(n, g, CC<float>(z), C<float>(r));
    return cudaGetLastError();
}

cudaError_t adj_outputs(bool dbl, int64_t m, int64_t n, const void* q, const void* z, const void* t,
                        const void* D, const void* l1, double* dlam, double* db, double* dA, int64_t ld_dA,
                        cudaStream_t s) {
    if (dlam) {
        if (dbl) adj_lambda_kernel<double><<<1, 1024, 0, s>>>(n, CC<double>(q), CC<double>(z), dlam);
        else adj_lambda_kernel<float><<<1, 1024, 0, s>>>(n, CC<float>(q), CC<float>(z), dlam);
    }
    const int gm = grid_for(m, VT_THREADS, 2048);
    if (db) {
        if (dbl) adj_db_kernel<double><<<gm, VT_THREADS, 0, s>>>(m, CC<double>(t), CC<double>(D), db);
        else adj_db_kernel<float><<<gm, VT_THREADS, 0, s>>>(m, CC<float>(t), CC<float>(D), db);
    }
    if (dA) {
        const int ga = grid_for(m * n, VT_THREADS, 8192);
        if (dbl)
            adj_da_kernel<double><<<ga, VT_THREADS, 0, s>>>(m, n, CC<double>(l1), CC<double>(q), CC<double>(D),
                                                            CC<double>(t), CC<double>(z), dA, ld_dA);
        else
            adj_da_kernel<float><<<ga, VT_THREADS, 0, s>>>(m, n, CC<float>(l1), CC<float>(q), CC<float>(D),
                                                           CC<float>(t), CC<float>(z), dA, ld_dA);
    }
    return cudaGetLastError();
}

}  // namespace genios
