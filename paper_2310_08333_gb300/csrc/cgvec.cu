// Vector work of the preconditioned CG iteration (§2.1, preconditioner Eq. (10)).
//
// Per iteration, after the fused Hv pass has left its per-CTA partial sums P (G x n):
//   cgv_q       (all SMs)   q = sum_b P[b] + nu p; per-block partials of p^T q and of U^T q.
//   cgv_kernel  (1 cluster) alpha = r^T z / p^T q; delta += alpha p; r -= alpha q; ||r||^2;
//                           w = U^T r by the recurrence w <- w - alpha U^T q; stop test;
//                           c_i = ((lam_s + nu) / (lam_i + nu) - 1) w_i  (Eq. (10));
//                           r^T z = ||r||^2 + sum_i c_i w_i (no pass over z); beta; and, inside
//                           the CUDA graph, the loop condition.
//   cgv_p       (all SMs)   z = r + U c;  p = z + beta p.
// The cluster owns a slice of every n-vector per CTA and reduces its scalars and s-vectors
// through distributed shared memory; the passes over U (n x s) run on all SMs.  Every sum is
// taken in a fixed order, and the cluster-wide sums are formed identically by every CTA, so the
// scalars agree bit for bit across the cluster and from run to run.
// The start of a solve (cgv_r0, then the cluster kernel in start mode, then cgv_p) forms the
// right-hand side of the step form of Eq. (7), w = U^T r directly, and p = z = P^{-1} r.
#include "common.cuh"
#include "internal.h"

#include <cooperative_groups.h>

namespace genios {

namespace cgx = cooperative_groups;

constexpr int CGV_THREADS = 512;
constexpr int CGV_ROWS = 32;          // rows of an n-vector per block of the all-SM kernels
constexpr int CGV_BT = 256;           // threads of the all-SM kernels
constexpr int CGV_STRIDE = 129;       // doubles per block partial: [0] scalar, [1 + c] s-vector
constexpr int RPT = 3;                // vector rows per thread of the cluster step (n <= 3 * 512 * CL)
constexpr int UNR = 12;               // block partials per thread of the cluster step (nb <= 48 CL)

int cgv_blocks(int64_t n) { return (int)((n + CGV_ROWS - 1) / CGV_ROWS); }
// the U^T r partials of cgv_p follow the cgv_q / cgv_r0 partials in the same buffer
static inline size_t part_r_offset(int nb) { return ((size_t)nb * CGV_STRIDE + 31) & ~size_t(31); }

// Block-wide sum of NV values of type T (float in float32 mode: this part's float64 pipe is
// narrow and the CG scalars need no more than float32), broadcast to every thread.
template <typename T, int NV>
GENIOS_DEV void bsum(T (&v)[NV]) {
    __shared__ T sh[32 * NV];
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
        const T t = lane < nw ? sh[k * 32 + lane] : T(0);
        v[k] = warp_sum(t);
    }
    __syncthreads();
}

// Block partial of U^T v over the block's 32 rows (v staged in shared memory), written with the
// block's scalar partial to part[blockIdx.x * 129 ...].  Threads: column c = t % 128, row half
// h = t / 128.
template <typename VT>
GENIOS_DEV void ut_partial(const VT* U, int sk, const VT* vsh, int64_t j0, int rows, VT scalar,
                           double* part) {
    __shared__ VT half1[128];
    const int t = threadIdx.x, c = t & 127, h = t >> 7;
    VT acc = VT(0);
    if (c < sk) {
        VT a = VT(0);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = h * 16 + k;
            if (i < rows) a = fma(U[(j0 + i) * sk + c], vsh[i], a);
        }
        acc = a;
    }
    if (h == 1) half1[c] = acc;
    __syncthreads();
    double* out = part + (size_t)blockIdx.x * CGV_STRIDE;
    if (h == 0 && c < sk) out[1 + c] = (double)(acc + half1[c]);
    if (t == 0) out[0] = (double)scalar;
}

// start: u <- u_scale u; r = -(g + rho (x - z + u)); delta = 0; partials of ||r||^2 and U^T r
template <typename VT>
__global__ void __launch_bounds__(CGV_BT) cgv_r0_kernel(int64_t n, const VT* g, const VT* x, const VT* z, VT* u,
                                                        double rho, double u_scale, VT* r, VT* delta,
                                                        const VT* U, int sk, double* part) {
    __shared__ VT rsh[CGV_ROWS];
    const int64_t j0 = (int64_t)blockIdx.x * CGV_ROWS;
    const int rows = (int)min((int64_t)CGV_ROWS, n - j0);
    VT rr = VT(0);
    if (threadIdx.x < CGV_ROWS) {
        VT rj = VT(0);
        if (threadIdx.x < rows) {
            const int64_t j = j0 + threadIdx.x;
            const VT uj = u[j] * (VT)u_scale;
            u[j] = uj;
            rj = -(g[j] + (VT)rho * (x[j] - z[j] + uj));
            r[j] = rj;
            delta[j] = VT(0);
            rr = rj * rj;
        }
        rsh[threadIdx.x] = rj;
    }
    VT v[1] = {rr};
    bsum<VT, 1>(v);   // its barriers also publish rsh
    ut_partial<VT>(U, sk, rsh, j0, rows, v[0], part);
}

// iteration: q = sum_b P[b] + nu p; partials of p^T q and U^T q
template <typename VT>
__global__ void __launch_bounds__(CGV_BT) cgv_q_kernel(const VT* P, int G, int64_t ldp, int64_t n, const VT* p,
                                                       VT* q, const VT* U, int sk, double* part,
                                                       const DevState* S, const VT* mask) {
    if (S->cg_done) return;
    __shared__ VT sh[8][33];
    __shared__ VT qsh[CGV_ROWS];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * CGV_ROWS;
    const int64_t j = j0 + tx;
    const int rows = (int)min((int64_t)CGV_ROWS, n - j0);
    VT a0 = VT(0), a1 = VT(0);
    if (j < n) {
        int b = ty;
        for (; b + 8 < G; b += 16) {
            a0 += P[(int64_t)b * ldp + j];
            a1 += P[(int64_t)(b + 8) * ldp + j];
        }
        for (; b < G; b += 8) a0 += P[(int64_t)b * ldp + j];
    }
    sh[ty][tx] = a0 + a1;
    __syncthreads();
    VT pq = VT(0);
    if (ty == 0) {
        VT qj = VT(0);
        if (j < n) {
            VT s = VT(0);
#pragma unroll
            for (int k = 0; k < 8; ++k) s += sh[k][tx];
            const VT pj = p[j];
            qj = s + (VT)S->nu * pj;
            if (mask != nullptr && mask[j] == VT(0)) qj = VT(0);   // operator restricted to the mask
            q[j] = qj;
            pq = pj * qj;
        }
        qsh[tx] = qj;
    }
    VT v[1] = {pq};
    bsum<VT, 1>(v);
    ut_partial<VT>(U, sk, qsh, j0, rows, v[0], part);
}

// the cluster step (start or iteration)
template <typename VT>
struct CgvArgs {
    int mode;   // 0: start of a solve, 1: one iteration
    int64_t n;
    int sk;
    double nu, tol;   // start
    int cg_max;       // start
    const VT* q;
    VT* r; VT* delta; const VT* p;
    const double* lam;
    const double* part;     // cgv_q (iteration) or cgv_r0 (start) block partials
    const double* part_r;   // cgv_p block partials of U^T r of the current residual
    int nb;
    DevState* S;
    unsigned long long cond;
    int use_cond, timed;
};

template <typename VT>
__global__ void __launch_bounds__(CGV_THREADS, 1) cgv_kernel(CgvArgs<VT> a) {
    cgx::cluster_group cluster = cgx::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int tid = threadIdx.x;
    using AT = VT;   // accumulation type: float in float32 mode
    __shared__ AT mypart[CGV_STRIDE];   // [0] ||r_slice||^2, [1 + c] this CTA's share of U^T (q or r)
    __shared__ AT tot[CGV_STRIDE];
    __shared__ AT grp[4][128];
    __shared__ AT lamsh[128];
    DevState* S = a.S;
    const int sk = a.sk;
    // device state of the previous launches, read once; this launch writes it only after its
    // last cluster barrier, when every CTA has read it
    const int done_in = a.mode == 1 ? S->cg_done : 0;
    const AT rz_old = (AT)S->rz, nu_s = (AT)S->nu, tol_s = (AT)S->tol, rhs2_in = (AT)S->rhs2;
    const int cgmax_s = S->cg_max, it_in = S->cg_it;
    if (tid < sk) lamsh[tid] = (AT)a.lam[tid];
    if (done_in) {
        if (a.use_cond && rank == 0 && tid == 0) cudaGraphSetConditional(a.cond, 0u);
        return;
    }
    const AT nu = a.mode == 1 ? nu_s : (AT)a.nu;
    const AT tol = a.mode == 1 ? tol_s : (AT)a.tol;
    const int cg_max = a.mode == 1 ? cgmax_s : a.cg_max;

    // Every global load of this step is issued here, before any reduction, so that the step
    // costs one memory round trip: the block partials of p^T q, this CTA's rows of the vectors,
    // and this CTA's share of the U^T q / U^T r block partials.
    const int64_t j0 = a.n * rank / CL, j1 = a.n * (rank + 1) / CL;
    VT pv[RPT], qv[RPT], rv[RPT], dv[RPT];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        const int64_t j = j0 + tid + (int64_t)t * CGV_THREADS;
        pv[t] = qv[t] = rv[t] = dv[t] = VT(0);
        if (j < j1) {
            rv[t] = a.r[j];
            if (a.mode == 1) {
                pv[t] = a.p[j];
                qv[t] = a.q[j];
                dv[t] = a.delta[j];
            }
        }
    }
    AT pqv = AT(0);
    if (a.mode == 1)
        for (int b = tid; b < a.nb; b += CGV_THREADS) pqv += (AT)a.part[(size_t)b * CGV_STRIDE];
    const int c = tid & 127, g4 = tid >> 7;
    const int b0 = (int)((int64_t)a.nb * rank / CL), b1 = (int)((int64_t)a.nb * (rank + 1) / CL);
    AT vq[UNR], vr[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
        const int bb = b0 + g4 + 4 * u;
        const bool ok = c < sk && bb < b1;
        vq[u] = ok ? (AT)a.part[(size_t)bb * CGV_STRIDE + 1 + c] : AT(0);
        vr[u] = (ok && a.mode == 1) ? (AT)a.part_r[(size_t)bb * CGV_STRIDE + 1 + c] : AT(0);
    }

    // alpha from the block partials of p^T q (same order in every CTA)
    AT pq = AT(0), alpha = AT(0);
    if (a.mode == 1) {
        AT v[1] = {pqv};
        bsum<AT, 1>(v);
        pq = v[0];
        alpha = pq > AT(0) ? rz_old / pq : AT(0);
    }

    // this CTA's rows: delta += alpha p, r -= alpha q, ||r||^2
    AT rr_loc = AT(0);
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        const int64_t j = j0 + tid + (int64_t)t * CGV_THREADS;
        if (j < j1) {
            VT rj = rv[t];
            if (a.mode == 1) {
                a.delta[j] = dv[t] + (VT)alpha * pv[t];
                rj = rv[t] - (VT)alpha * qv[t];
                a.r[j] = rj;
            }
            rr_loc += rj * rj;
        }
    }
    // this CTA's share of the block partials: start: U^T r; iteration: U^T r_old - alpha U^T q
    // (the direct U^T r of the previous residual comes from cgv_p, so the recurrence spans one step)
    {
        AT sacc = AT(0);
#pragma unroll
        for (int u = 0; u < UNR; ++u) sacc += a.mode == 1 ? vr[u] - alpha * vq[u] : vq[u];
        grp[g4][c] = sacc;
    }
    {
        AT v[1] = {rr_loc};
        bsum<AT, 1>(v);   // its barriers also publish grp
        if (tid == 0) mypart[0] = v[0];
    }
    if (tid < sk) mypart[1 + tid] = (grp[0][tid] + grp[1][tid]) + (grp[2][tid] + grp[3][tid]);
    cluster.sync();

    // cluster totals, summed over ranks in order by every CTA
    for (int k = tid; k <= sk; k += CGV_THREADS) {
        AT vals[16];   // all remote loads in flight at once; zeros past CL leave the sum exact
#pragma unroll
        for (int q = 0; q < 16; ++q) vals[q] = q < CL ? cluster.map_shared_rank(mypart, q)[k] : AT(0);
        AT s = AT(0);
#pragma unroll
        for (int q = 0; q < 16; ++q) s += vals[q];
        tot[k] = s;
    }
    __syncthreads();
    const AT rr = tot[0];
    const AT ls = sk > 0 ? lamsh[sk - 1] : AT(0);
    AT rzc = AT(0);
    if (tid < sk) {
        const AT w = tot[1 + tid];
        const AT cw = ((ls + nu) / (lamsh[tid] + nu) - AT(1)) * w;
        rzc = cw * w;
        if (rank == 0) S->cgc[tid] = (double)cw;
    }
    AT v[1] = {rzc};
    bsum<AT, 1>(v);
    const AT rz = rr + v[0];
    const AT beta = a.mode == 1 && rz_old > AT(0) ? rz / rz_old : AT(0);
    cluster.sync();   // no CTA leaves while another still reads its mypart

    if (rank == 0 && tid == 0) {
        if (a.mode == 0) {
            S->rhs2 = rr;
            S->rr = rr;
            S->nu = nu;
            S->tol = tol;
            S->cg_it = 0;
            S->cg_max = cg_max;
            S->cg_done = rr > AT(0) ? 0 : 1;
            S->cg_first = 0;
            S->cg_guard = 0;
            S->hv_t0 = ~0ull;
            S->hv_t1 = 0ull;
            S->alpha = 0.0;
            S->pq = 0.0;
            S->beta = 0.0;
            S->rz = rz;
        } else {
            const int it = it_in + 1;
            const bool done = !(pq > AT(0)) || rr <= tol * tol * rhs2_in || it >= cg_max;
            S->pq = pq;
            S->alpha = alpha;
            S->rr = rr;
            S->cg_it = it;
            S->cg_done = done ? 1 : 0;
            S->beta = beta;
            S->rz = rz;
            if (a.timed && S->hv_t1 > S->hv_t0) {   // fold this iteration's Hv device time
                S->hv_ns += (double)(S->hv_t1 - S->hv_t0);
                S->hv_count += 1;
            }
            S->hv_t0 = ~0ull;
            S->hv_t1 = 0ull;
            const int guard = ++S->cg_guard;
            const int cap = cg_max < 10000 ? cg_max : 10000;   // hard bound on the device loop
            if (a.use_cond) cudaGraphSetConditional(a.cond, (!done && guard < cap + 2) ? 1u : 0u);
        }
    }
}

// z = r + U c and p = z + beta p (beta = 0: p = z), plus the block partials of U^T r for the next
// iteration's w.  One warp per row, four columns per lane.
template <typename VT>
__global__ void __launch_bounds__(CGV_BT) cgv_p_kernel(int64_t n, const VT* r, VT* p, const VT* U, int sk,
                                                       double* part_r, const DevState* S, const VT* mask) {
    if (S->cg_done) return;
    __shared__ VT csh[128];
    __shared__ VT ush[CGV_BT / 32][128];
    for (int c = threadIdx.x; c < 128; c += CGV_BT) csh[c] = c < sk ? (VT)S->cgc[c] : VT(0);
    const VT beta = (VT)S->beta;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * CGV_ROWS;
    VT cl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) cl[k] = csh[lane + 32 * k];
    constexpr int RPW = CGV_ROWS / (CGV_BT / 32);   // rows per warp
    VT acc[RPW], rv[RPW];
    VT ur[4] = {VT(0), VT(0), VT(0), VT(0)};
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
        acc[t] = VT(0);
        const int64_t j = j0 + wid * RPW + t;
        rv[t] = j < n ? r[j] : VT(0);
        if (j < n && sk > 0) {
            const VT* Uj = U + j * sk;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = lane + 32 * k;
                if (c < sk) {
                    const VT u = Uj[c];
                    acc[t] = fma(u, cl[k], acc[t]);
                    ur[k] = fma(u, rv[t], ur[k]);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < RPW; ++t) acc[t] = warp_sum(acc[t]);
    if (lane < RPW) {
        VT mine = acc[0];
#pragma unroll
        for (int t = 1; t < RPW; ++t)
            if (lane == t) mine = acc[t];
        const int64_t j = j0 + wid * RPW + lane;
        if (j < n) {
            VT rj = rv[0];
#pragma unroll
            for (int t = 1; t < RPW; ++t)
                if (lane == t) rj = rv[t];
            const VT zj = rj + mine;
            if (mask != nullptr && mask[j] == VT(0)) p[j] = VT(0);   // preconditioner restricted too
            else p[j] = beta != VT(0) ? zj + beta * p[j] : zj;
        }
    }
    if (sk > 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) ush[wid][lane + 32 * k] = ur[k];
        __syncthreads();
        double* out = part_r + (size_t)blockIdx.x * CGV_STRIDE;
        for (int c = threadIdx.x; c < sk; c += CGV_BT) {
            VT s = VT(0);
#pragma unroll
            for (int w = 0; w < CGV_BT / 32; ++w) s += ush[w][c];
            out[1 + c] = (double)s;
        }
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <typename VT>
static CgvPlan plan_vt(int64_t n, int sk) {
    CgvPlan p{};
    p.ok = false;
    if (sk < 0 || sk > 128 || n < 1) return p;
    cudaFuncSetAttribute(cgv_kernel<VT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cl : {16, 8}) {
        if ((n + cl - 1) / cl > (int64_t)RPT * CGV_THREADS || (cgv_blocks(n) + cl - 1) / cl > 4 * UNR) continue;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(CGV_THREADS);
        cfg.dynamicSmemBytes = 0;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, cgv_kernel<VT>, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        p.cl = cl;
        p.ok = true;
        return p;
    }
    return p;
}

CgvPlan cgv_plan(bool dbl, int64_t n, int sk) { return dbl ? plan_vt<double>(n, sk) : plan_vt<float>(n, sk); }

template <typename VT>
static cudaError_t launch_cluster(const CgvPlan& pl, const CgvArgs<VT>& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(pl.cl);
    cfg.blockDim = dim3(CGV_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = pl.cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cgv_kernel<VT>, a);
}

template <typename VT>
static cudaError_t start_vt(const CgvPlan& pl, int64_t n, const void* g, const void* x, const void* z, void* u,
                            double rho, double u_scale, double nu, double tol, int cg_max, void* r, void* delta,
                            void* p, const void* U, int sk, const double* lam, DevState* S, double* part,
                            const void* mask, cudaStream_t s) {
    const int nb = cgv_blocks(n);
    cgv_r0_kernel<VT><<<nb, CGV_BT, 0, s>>>(n, static_cast<const VT*>(g), static_cast<const VT*>(x),
                                            static_cast<const VT*>(z), static_cast<VT*>(u), rho, u_scale,
                                            static_cast<VT*>(r), static_cast<VT*>(delta), static_cast<const VT*>(U),
                                            sk, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CgvArgs<VT> a{};
    a.mode = 0;
    a.n = n;
    a.sk = sk;
    a.nu = nu;
    a.tol = tol;
    a.cg_max = cg_max;
    a.r = static_cast<VT*>(r);
    a.delta = static_cast<VT*>(delta);
    a.p = static_cast<const VT*>(p);
    a.lam = lam;
    a.part = part;
    a.part_r = part + part_r_offset(nb);
    a.nb = nb;
    a.S = S;
    e = launch_cluster(pl, a, s);
    if (e != cudaSuccess) return e;
    cgv_p_kernel<VT><<<nb, CGV_BT, 0, s>>>(n, static_cast<const VT*>(r), static_cast<VT*>(p),
                                           static_cast<const VT*>(U), sk, part + part_r_offset(nb), S,
                                           static_cast<const VT*>(mask));
    return cudaGetLastError();
}

cudaError_t cgv_start(bool dbl, const CgvPlan& pl, int64_t n, const void* g, const void* x, const void* z,
                      void* u, double rho, double u_scale, double nu, double tol, int cg_max, void* r,
                      void* delta, void* p, const void* U, int sk, const double* lam, DevState* S,
                      double* part, const void* mask, cudaStream_t s) {
    if (!pl.ok || sk > 128) return cudaErrorInvalidValue;
    return dbl ? start_vt<double>(pl, n, g, x, z, u, rho, u_scale, nu, tol, cg_max, r, delta, p, U, sk, lam, S,
                                  part, mask, s)
               : start_vt<float>(pl, n, g, x, z, u, rho, u_scale, nu, tol, cg_max, r, delta, p, U, sk, lam, S,
                                 part, mask, s);
}

cudaError_t cgv_q(bool dbl, const void* P, int G, int64_t ldp, int64_t n, const void* p, void* q, const void* U,
                  int sk, double* part, const DevState* S, const void* mask, cudaStream_t s) {
    const int nb = cgv_blocks(n);
    if (dbl)
        cgv_q_kernel<double><<<nb, CGV_BT, 0, s>>>(static_cast<const double*>(P), G, ldp, n,
                                                   static_cast<const double*>(p), static_cast<double*>(q),
                                                   static_cast<const double*>(U), sk, part, S,
                                                   static_cast<const double*>(mask));
    else
        cgv_q_kernel<float><<<nb, CGV_BT, 0, s>>>(static_cast<const float*>(P), G, ldp, n,
                                                  static_cast<const float*>(p), static_cast<float*>(q),
                                                  static_cast<const float*>(U), sk, part, S,
                                                  static_cast<const float*>(mask));
    return cudaGetLastError();
}

template <typename VT>
static cudaError_t iter_vt(const CgvPlan& pl, int64_t n, const void* q, void* r, void* delta, void* p,
                           const void* U, int sk, const double* lam, DevState* S, double* part,
                           unsigned long long cond, int use_cond, int timed, const void* mask, cudaStream_t s) {
    const int nb = cgv_blocks(n);
    CgvArgs<VT> a{};
    a.mode = 1;
    a.n = n;
    a.sk = sk;
    a.q = static_cast<const VT*>(q);
    a.r = static_cast<VT*>(r);
    a.delta = static_cast<VT*>(delta);
    a.p = static_cast<const VT*>(p);
    a.lam = lam;
    a.part = part;
    a.part_r = part + part_r_offset(nb);
    a.nb = nb;
    a.S = S;
    a.cond = cond;
    a.use_cond = use_cond;
    a.timed = timed;
    cudaError_t e = launch_cluster(pl, a, s);
    if (e != cudaSuccess) return e;
    cgv_p_kernel<VT><<<nb, CGV_BT, 0, s>>>(n, static_cast<const VT*>(r), static_cast<VT*>(p),
                                           static_cast<const VT*>(U), sk, part + part_r_offset(nb), S,
                                           static_cast<const VT*>(mask));
    return cudaGetLastError();
}

cudaError_t cgv_iter(bool dbl, const CgvPlan& pl, int64_t n, const void* q, void* r, void* delta, void* p,
                     const void* U, int sk, const double* lam, DevState* S, double* part,
                     unsigned long long cond, int use_cond, int timed, const void* mask, cudaStream_t s) {
    if (!pl.ok || sk > 128) return cudaErrorInvalidValue;
    return dbl ? iter_vt<double>(pl, n, q, r, delta, p, U, sk, lam, S, part, cond, use_cond, timed, mask, s)
               : iter_vt<float>(pl, n, q, r, delta, p, U, sk, lam, S, part, cond, use_cond, timed, mask, s);
}

}  // namespace genios
