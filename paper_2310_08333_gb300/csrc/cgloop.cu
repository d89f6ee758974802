// Persistent preconditioned CG (§2.1 with the Nystrom preconditioner of Eq. (10)): the whole CG
// solve of one x-subproblem in a single cooperative launch of one CTA per SM.
//
// Every CTA owns a contiguous block of rows of A (the Hv pass) and a contiguous slice of every
// n-vector (the vector work).  Per iteration, with grid-wide barriers (|) between the phases:
//   H  the fused pass y_b = A_b^T diag(d_b) A_b p over the CTA's rows (the rowpass consumer)
//      and p^T y_b (summed over the CTAs: p^T A^T diag(d) A p)
//   |  Q  pq = p^T H p + nu ||p||^2, alpha = r^T z / pq; on the slice: q = sum_b y_b + nu p,
//         delta += alpha p, r -= alpha q, and the slice's partials of ||r||^2 and U^T r
//   |  P  w = U^T r and ||r||^2 (sums of the partials, in the same order in every CTA), the stop
//         test, c_i = ((lam_s + nu) / (lam_i + nu) - 1) w_i, r^T z = ||r||^2 + c^T w, beta; on the
//         slice: p = r + U c + beta p and its share of ||p||^2
//   |  (next H)
// The start of the solve forms the step-form right-hand side of Eq. (7) on the slices (r, delta,
// u), then runs P with beta = 0.  All scalars come out bit-identical in every CTA, so every CTA
// takes the same branch at the stop test.  A producer warp per CTA streams the CTA's rows into a
// ring of shared-memory stages without pause across iterations: the next pass's first stages load
// while the vector phases run.
// Every wait is bounded (mbarriers and the grid barrier): on expiry the CTA records a fault in
// DevState::cg_fault, which makes the other CTAs leave at their next barrier, its producer waits
// for the copies it issued, and the kernel returns.
#include "rowpass_core.cuh"
#include "devloop.cuh"

#include <algorithm>

namespace genios {

constexpr int CGL_ST = 132;          // stride of a CTA's partial: [0] scalar, [1 + c] s-vector
constexpr int CGL_SLICE_MAX = 1024;  // vector entries per CTA
constexpr size_t CGL_SMEM_BUDGET = 196 * 1024;   // ring stages + mbarriers + row-total scratch


GENIOS_DEV unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
GENIOS_DEV void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
GENIOS_DEV unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared state of a CTA.  The scalars are computed identically by all consumer threads and
// stored by thread 0; they live here, not in registers, so that nothing but the Hv pass's own
// values is live across the Hv phase.
template <typename VT>
struct CglShared {
    VT vsl[CGL_SLICE_MAX];      // the slice of r (start, Q)
    VT grp[4][CGL_ST];
    VT tot[CGL_ST];
    VT csh[128];                // preconditioner coefficients c
    VT lamsh[128];
    VT colsum[8][64];
    VT red16[RP_CTHREADS * (16 / sizeof(VT))];   // 16-byte partial sums of the partial-row reduction
    VT sh16[RP_CWARPS];
    double dsh16[RP_CWARPS];     // csum of float64 values
    VT rz_old, rhs2, rr, rz, alpha, beta, pq;
    unsigned long long t_start, t_mark;
    int64_t j0, r0, nrows;      // the slice and the row block
    int ns, nstage_work, it, start;
    unsigned epoch;             // grid barriers passed (thread 0)
    int32_t stop;               // set by the consumers when they leave; read by the producer
    double rho, u_scale, nu, tol, zu_rho, zu_lam1;   // this x-step's parameters (arguments, or DevLoop)
};

// Grid barrier among the consumer threads of all CTAs (co-resident: cooperative launch).  The
// counter only grows during a launch; the k-th barrier waits for k * gridDim.x arrivals.
// Returns false, the same in every consumer thread of the CTA, on a timeout or another CTA's fault.
template <typename VT>
GENIOS_DEV bool grid_sync(const CgLoopArgs& a, CglShared<VT>& sh) {
    named_bar_sync(1, RP_CTHREADS);
    bool bad = false;
    if (threadIdx.x == 0) {
        const unsigned target = ++sh.epoch * gridDim.x;
        int32_t* fault = &a.S->cg_fault;
        // release: this CTA's writes before the barrier above; acquire: the other CTAs' writes
        red_release_add_u32(a.bar, 1u);
        const long long t0 = clock64();
        while ((int)(ld_acquire_u32(a.bar) - target) < 0) {
            if (*reinterpret_cast<volatile int32_t*>(fault) != 0) { bad = true; break; }
            if (clock64() - t0 > a.rp.wait_limit) {
                atomicCAS(reinterpret_cast<int*>(fault), 0, 2);
                bad = true;
                break;
            }
        }
    }
    return !named_bar_or(2, RP_CTHREADS, bad);
}

// Sum of one value over the 512 consumer threads, in a fixed order; valid in every one of them.
template <typename VT>
GENIOS_DEV VT csum(VT v, VT* sh16) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh16[threadIdx.x >> 5] = v;
    named_bar_sync(1, RP_CTHREADS);
    VT t = VT(0);
#pragma unroll
    for (int w = 0; w < RP_CWARPS; ++w) t += sh16[w];
    named_bar_sync(1, RP_CTHREADS);
    return t;
}

// sum over bb = h, h + step, ... < G of X[bb * ld + k], eight loads in flight, in a fixed order
template <typename VT>
GENIOS_DEV VT strided_sum(const VT* X, size_t ld, int k, int h, int step, int G) {
    VT acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = VT(0);
    int bb = h;
    for (; bb + 7 * step < G; bb += 8 * step) {
        VT v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(X + (size_t)(bb + u * step) * ld + k);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += v[u];
    }
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (bb + u * step < G) acc[u] += __ldcg(X + (size_t)(bb + u * step) * ld + k);
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// Rows jb, jb + 4, ..., jb + 60 of the CTA's slice of U at column threadIdx.x % 128 (zero past the
// slice or past column s).
template <typename VT>
GENIOS_DEV void slice_u_rows(const VT* U, int sk, int64_t j0, int ns, int jb, VT (&u)[16]) {
    const int c = threadIdx.x & 127;
#pragma unroll
    for (int t = 0; t < 16; ++t) u[t] = (c < sk && jb + 4 * t < ns) ? U[(j0 + jb + 4 * t) * sk + c] : VT(0);
}

// The CTA's partial [scalar, U_slice^T v_slice] into out[0 .. sk].  vsl: the slice of v in shared
// memory (published by the caller's last barrier); U rows j0 .. j0 + ns - 1, the first 16 of the
// thread's rows (jb = threadIdx.x / 128) already in u0.
template <typename VT>
GENIOS_DEV void slice_partial(const VT* U, int sk, int64_t j0, int ns, VT scalar, VT* out, CglShared<VT>& sh,
                              const VT (&u0)[16]) {
    const int tid = threadIdx.x, c = tid & 127, h = tid >> 7;
    VT acc[4] = {VT(0), VT(0), VT(0), VT(0)};
    if (c < sk) {
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (h + 4 * t < ns) acc[t & 3] = fma(u0[t], sh.vsl[h + 4 * t], acc[t & 3]);
        for (int jb = h + 64; jb < ns; jb += 64) {
            VT u[16];
            slice_u_rows(U, sk, j0, ns, jb, u);
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (jb + 4 * t < ns) acc[t & 3] = fma(u[t], sh.vsl[jb + 4 * t], acc[t & 3]);
        }
    }
    sh.grp[h][c] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    const VT tot = csum(scalar, sh.sh16);   // its barriers also publish grp
    if (tid < sk) out[1 + tid] = (sh.grp[0][tid] + sh.grp[1][tid]) + (sh.grp[2][tid] + sh.grp[3][tid]);
    if (tid == 0) out[0] = tot;
}

// start: u <- u_scale u; r = -(g + rho (x - z + u)); delta = 0 on the slice; partials of ||r||^2, U^T r
template <typename VT>
GENIOS_DEV void cg_start(const CgLoopArgs& a, CglShared<VT>& sh) {
    const int tid = threadIdx.x;
    const int64_t j0 = sh.j0;
    const int ns = sh.ns;
    const VT* g = static_cast<const VT*>(a.g);
    const VT* x = static_cast<const VT*>(a.x);
    const VT* z = static_cast<const VT*>(a.z);
    VT* u = static_cast<VT*>(a.u);
    VT* r = static_cast<VT*>(a.r);
    VT* delta = static_cast<VT*>(a.delta);
    VT u0[16];
    slice_u_rows(static_cast<const VT*>(a.U), a.sk, j0, ns, tid >> 7, u0);
    VT rr = VT(0);
    for (int jj = tid; jj < ns; jj += RP_CTHREADS) {
        const int64_t j = j0 + jj;
        const VT uj = u[j] * (VT)sh.u_scale;
        u[j] = uj;
        const VT rj = -(g[j] + (VT)sh.rho * (x[j] - z[j] + uj));
        r[j] = rj;
        delta[j] = VT(0);
        sh.vsl[jj] = rj;
        rr += rj * rj;
    }
    named_bar_sync(1, RP_CTHREADS);
    slice_partial<VT>(static_cast<const VT*>(a.U), a.sk, j0, ns, rr,
                      static_cast<VT*>(a.part) + (size_t)blockIdx.x * CGL_ST, sh, u0);
}

// Rows jb + 16 t (t < 4) of the CTA's slice for the new direction: U row entries at columns
// lane + 32 k (zero past s), and in lane 0 r_j and p_j.
template <typename VT>
GENIOS_DEV void dir_rows_load(const CgLoopArgs& a, int64_t j0, int ns, int jb, VT (&ur)[4][4], VT (&rv)[4],
                              VT (&pv)[4]) {
    const int lane = threadIdx.x & 31, sk = a.sk;
    const VT* U = static_cast<const VT*>(a.U);
    const VT* r = static_cast<const VT*>(a.r);
    const VT* p = static_cast<const VT*>(a.p);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int jj = jb + t * RP_CWARPS;
        const int64_t j = j0 + jj;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            ur[t][k] = (jj < ns && c < sk) ? U[j * sk + c] : VT(0);
        }
        rv[t] = (jj < ns && lane == 0) ? r[j] : VT(0);
        pv[t] = (jj < ns && lane == 0) ? p[j] : VT(0);
    }
}

// P: w = U^T r and ||r||^2 from the partials, the stop test, c, r^T z, beta, and on the slice
// p = r + U c + beta p.  Returns false when the solve is done.
template <typename VT>
GENIOS_DEV bool cg_direction(const CgLoopArgs& a, CglShared<VT>& sh) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x, sk = a.sk;
    const VT nu = (VT)sh.nu;
    const VT* partW = static_cast<const VT*>(a.part);
    const int64_t j0 = sh.j0;
    const int ns = sh.ns;
    {   // sum of the G partial rows [||r||^2, U^T r]: 16-byte columns x row groups, 8 loads in flight
        constexpr int VW = 16 / sizeof(VT);
        const int nq = (sk + 1 + VW - 1) / VW;
        const int nh = min(G, RP_CTHREADS / nq);
        const int q = tid % nq, h = tid / nq;
        if (h < nh) {
            VT acc[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) acc[e] = VT(0);
            for (int bb = h; bb < G; bb += 8 * nh) {
                uint4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = bb + u * nh < G ? __ldcg(reinterpret_cast<const uint4*>(partW + (size_t)(bb + u * nh) * CGL_ST) + q)
                                           : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    VT f[VW];
                    decode_chunk(v[u], f);
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[e] += f[e];
                }
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) sh.red16[(h * nq + q) * VW + e] = acc[e];
        }
        named_bar_sync(1, RP_CTHREADS);
        if (tid <= sk) {
            VT t = VT(0);
            for (int hh = 0; hh < nh; ++hh) t += sh.red16[hh * nq * VW + tid];
            sh.tot[tid] = t;
        }
        named_bar_sync(1, RP_CTHREADS);
    }
    const VT rr = sh.tot[0];
    const VT ls = sk > 0 ? sh.lamsh[sk - 1] : VT(0);
    VT cw = VT(0);
    if (tid < sk) {
        const VT w = sh.tot[1 + tid];
        const VT c = ((ls + nu) / (sh.lamsh[tid] + nu) - VT(1)) * w;
        sh.csh[tid] = c;
        cw = c * w;
    } else if (tid < 128) {
        sh.csh[tid] = VT(0);
    }
    const bool start = sh.start != 0;
    const VT rz_old = sh.rz_old;
    VT rhs2 = sh.rhs2;
    int it = sh.it;
    const VT rz = rr + csum(cw, sh.sh16);   // its barriers also publish csh
    bool done;
    if (start) {
        rhs2 = rr;
        done = !(rr > VT(0));
    } else {
        ++it;
        done = rr <= (VT)sh.tol * (VT)sh.tol * rhs2 || it >= a.cg_max;
    }
    const VT beta = (!start && rz_old > VT(0)) ? rz / rz_old : VT(0);
    if (!done) {
        const VT* mask = static_cast<const VT*>(a.mask);
        VT* p = static_cast<VT*>(a.p);
        VT cl[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cl[k] = sh.csh[lane + 32 * k];
        VT pp = VT(0);
        for (int jb = wid; jb < ns; jb += 4 * RP_CWARPS) {   // four rows per warp in flight
            VT ur[4][4], rv[4], pv[4];
            dir_rows_load(a, j0, ns, jb, ur, rv, pv);
            VT acc[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                acc[t] = VT(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[t] = fma(ur[t][k], cl[k], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[t] = warp_sum(acc[t]);
            if (lane == 0) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int jj = jb + t * RP_CWARPS;
                    if (jj < ns) {
                        const int64_t j = j0 + jj;
                        VT pj = rv[t] + acc[t];
                        if (!start) pj += beta * pv[t];
                        if (mask != nullptr && mask[j] == VT(0)) pj = VT(0);
                        p[j] = pj;
                        pp += pj * pj;
                    }
                }
            }
        }
        pp = csum(pp, sh.sh16);
        if (tid == 0) static_cast<VT*>(a.part)[(size_t)G * CGL_ST + G + blockIdx.x] = pp;
    }
    if (tid == 0) {   // every thread has read the old values (csum's barriers lie in between)
        sh.rr = rr;
        sh.rz = rz;
        sh.rhs2 = rhs2;
        sh.it = it;
        sh.beta = beta;
        sh.start = 0;
        if (!done) sh.rz_old = rz;
    }
    return !done;
}

// Q: pq = p^T H p + nu ||p||^2, alpha; on the slice q = sum_b y_b + nu p, delta += alpha p,
// r -= alpha q; partials of ||r||^2 and U^T r.  Returns false on a breakdown (pq <= 0).
template <typename VT>
GENIOS_DEV bool cg_step(const CgLoopArgs& a, CglShared<VT>& sh) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    const VT nu = (VT)sh.nu;
    VT* partW = static_cast<VT*>(a.part);
    const VT* partH = partW + (size_t)G * CGL_ST;
    const VT* partPP = partH + G;
    const int64_t j0 = sh.j0;
    const int ns = sh.ns;
    const VT* Pb = static_cast<const VT*>(a.rp.partial);
    const VT* mask = static_cast<const VT*>(a.mask);
    const VT* p = static_cast<const VT*>(a.p);
    VT* r = static_cast<VT*>(a.r);
    VT* delta = static_cast<VT*>(a.delta);
    const int64_t ldp = a.rp.ldp;
    VT u0[16];   // the first rows of U for the partial of U^T r, loaded with everything else
    slice_u_rows(static_cast<const VT*>(a.U), a.sk, j0, ns, tid >> 7, u0);
    VT rl = VT(0), pq = VT(0), alpha = VT(0);
    for (int cb = 0; cb < max(ns, 1); cb += 64) {   // at least once: pq is formed in every CTA
        // every load of the chunk at once: 8 row groups x 64 columns of the partials y_b, the
        // slice entries, and (first chunk, warp 0) the partials of p^T A^T D A p and ||p||^2
        const int c = tid & 63, h = tid >> 6;
        const bool col = cb + c < ns;
        VT sq = VT(0);
        for (int bb = h; bb < G; bb += 160) {
            VT v[20];
#pragma unroll
            for (int u = 0; u < 20; ++u) v[u] = (col && bb + 8 * u < G) ? __ldcg(Pb + (int64_t)(bb + 8 * u) * ldp + j0 + cb + c) : VT(0);
#pragma unroll
            for (int u = 0; u < 20; ++u) sq += v[u];
        }
        VT pj = VT(0), rj = VT(0), dj = VT(0);
        bool live = true;
        if (tid < 64 && cb + tid < ns) {
            const int64_t j = j0 + cb + tid;
            pj = p[j];
            rj = r[j];
            dj = delta[j];
            live = mask == nullptr || mask[j] != VT(0);
        }
        if (cb == 0 && wid == RP_CWARPS - 1) {
            VT ph = VT(0), ppp = VT(0);
            for (int bb = lane; bb < G; bb += 32) {
                ph += __ldcg(partH + bb);
                ppp += __ldcg(partPP + bb);
            }
            ph = warp_sum(ph);
            ppp = warp_sum(ppp);
            if (lane == 0) {
                sh.tot[0] = ph;
                sh.tot[1] = ppp;
            }
        }
        sh.colsum[h][c] = sq;
        named_bar_sync(1, RP_CTHREADS);
        pq = sh.tot[0] + nu * sh.tot[1];
        if (!(pq > VT(0))) break;   // uniform: every thread read the same pq
        alpha = sh.rz_old / pq;
        if (tid < 64 && cb + tid < ns) {
            const int64_t j = j0 + cb + tid;
            VT s2 = VT(0);
#pragma unroll
            for (int hh = 0; hh < 8; ++hh) s2 += sh.colsum[hh][tid];
            const VT qj = live ? s2 + nu * pj : VT(0);
            delta[j] = dj + alpha * pj;
            rj -= alpha * qj;
            r[j] = rj;
            sh.vsl[cb + tid] = rj;
            rl += rj * rj;
        }
        named_bar_sync(1, RP_CTHREADS);
    }
    if (!(pq > VT(0))) {   // breakdown (p = 0 or an indefinite operator): stop at the iterate
        if (tid == 0) sh.pq = pq;
        return false;
    }
    slice_partial<VT>(static_cast<const VT*>(a.U), a.sk, j0, ns, rl, partW + (size_t)blockIdx.x * CGL_ST, sh, u0);
    if (tid == 0) {
        sh.pq = pq;
        sh.alpha = alpha;
    }
    return true;
}

// The z/u update of §2.5 / Eq. (5) after the x-step, on the CTA's slice: x += delta,
// x_hat = alpha x + (1 - alpha) z, z = S_{lambda_1 / rho}(x_hat + u) (with a box: the projection of
// x_hat + u onto it), u += x_hat - z; and the norms
// ||x - z||^2, ||x||^2, ||z||^2, ||u||^2, ||z||_1, nnz(z) into DevState.  The CTA partials (float64)
// are summed in a fixed order by the last CTA to finish, so no grid barrier is needed.
template <typename VT>
GENIOS_DEV void zu_phase(const CgLoopArgs& a, CglShared<VT>& sh) {
    __shared__ double zsh[RP_CWARPS][6];
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    const int64_t j0 = sh.j0;
    const int ns = sh.ns;
    VT* x = static_cast<VT*>(a.zu_x);
    VT* z = static_cast<VT*>(a.zu_z);
    VT* u = static_cast<VT*>(a.u);
    const VT* delta = static_cast<const VT*>(a.delta);
    const double kappa = sh.zu_lam1 / sh.zu_rho;
    const double alpha = a.zu_alpha;
    const int box = a.zu_box;
    const VT lo = (VT)a.zu_lo, hi = (VT)a.zu_hi;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int jj = tid; jj < ns; jj += RP_CTHREADS) {
        const int64_t j = j0 + jj;
        const VT xj = x[j] + delta[j];
        x[j] = xj;
        const VT zj = z[j];
        const VT xh = (VT)alpha * xj + (VT)(1.0 - alpha) * zj;
        const VT vv = xh + u[j];
        VT zn;
        if (box) zn = vv < lo ? lo : vv > hi ? hi : vv;   // projection onto the box
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
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) zsh[wid][k] = v[k];
    named_bar_sync(1, RP_CTHREADS);
    double* zpart = a.zu_part;
    if (tid == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < RP_CWARPS; ++w)
#pragma unroll
            for (int k = 0; k < 6; ++k) t[k] += zsh[w][k];
#pragma unroll
        for (int k = 0; k < 6; ++k) zpart[(size_t)blockIdx.x * 6 + k] = t[k];
        __threadfence();
        last = atomicAdd(a.bar + 1, 1u) == (unsigned)(G - 1) ? 1 : 0;
    }
    named_bar_sync(1, RP_CTHREADS);
    if (!last) return;
    __threadfence();
    if (wid < 6) {   // warp k sums norm k over the CTAs in a fixed order
        double t = 0.0;
        for (int bb = lane; bb < G; bb += 32) t += __ldcg(zpart + (size_t)bb * 6 + wid);
        t = warp_sum(t);
        if (lane == 0) {
            DevState* S = a.S;
            if (wid == 0) S->rp2 = t;
            else if (wid == 1) S->x2 = t;
            else if (wid == 2) S->z2 = t;
            else if (wid == 3) S->u2 = t;
            else if (wid == 4) S->z1 = t;
            else S->nnz = t;
        }
    }
}

// The gradient finish after the fused gradient pass: g = the sum of the CTAs' partial rows plus
// lambda_2 x, the norms of grad_finish (||g + rho u||^2, ||rho u||^2, ||g||^2,
// ||(|A^T w| - lambda_1)_+||^2, ||x||_1, ||x||^2, max |A^T w|) and the loss sum, then the loop's
// decisions (phase a, and phase b when no KKT check is due) and the graph conditionals.  Every
// value is formed in grad_finish's order, bit for bit: a block of 32 columns (one per lane; the
// column sum over the CTAs' rows in eight interleaved classes, as column_sum does) ends in the
// block's butterfly sums; the last CTA to finish sums the blocks as grid_sum_max's
// last block does (256 threads, block t, t + 256, ... per thread, a butterfly within and across
// the 8 warps).
template <typename VT>
GENIOS_DEV void grad_finish_phase(const CgLoopArgs& a, CglShared<VT>& sh) {
    __shared__ int glast;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    DevLoop* L = a.loop;
    const double mu = L->lam2, rho = L->rho, lam1 = L->lam1;
    // k^gamma for the decisions (phase a makes this iteration k + 1), read now: its latency hides
    // behind the column sums
    const double kpow_next = tid == 0 ? loop_kpow(L, L->k + 1) : 0.0;
    const VT* P = static_cast<const VT*>(a.rp.partial);
    const int64_t ldp = a.rp.ldp, n = a.rp.n;
    const VT* x = static_cast<const VT*>(a.zu_x);
    const VT* u = static_cast<const VT*>(a.u);
    VT* g = static_cast<VT*>(a.g_out);
    const int nblk = (int)((n + 31) / 32);
    // two blocks of 32 columns at a time per CTA, eight warps each: warp q of a group forms the
    // column sums of class q (rows q, q + 8, ... in increasing order, loads issued ahead), the
    // group's first warp adds the classes 0..7 in order and finishes the columns
    // the class sums [2][8][32] doubles live in the slice buffer, free once the CG solve is over
    // (4 KB: 1024 floats or half of 1024 doubles), so that the kernel's static shared memory
    // stays within the device's limit beside the ring
    static_assert(sizeof(VT) * CGL_SLICE_MAX >= 2 * 8 * 32 * sizeof(double), "slice buffer too small");
    double (*csh)[8][32] = reinterpret_cast<double (*)[8][32]>(sh.vsl);
    const int grp = wid >> 3, q = wid & 7;
    for (int base = blockIdx.x * 2; base < nblk; base += G * 2) {   // uniform over the CTA
        const int blk = base + grp;
        const int64_t j = (int64_t)blk * 32 + lane;
        double accq = 0.0;
        if (blk < nblk && j < n) {
            for (int b0 = q; b0 < G; b0 += 64) {
                VT w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) w[t] = b0 + 8 * t < G ? __ldcg(P + (int64_t)(b0 + 8 * t) * ldp + j) : VT(0);
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (b0 + 8 * t < G) accq += (double)w[t];
            }
        }
        csh[grp][q][lane] = accq;
        named_bar_sync(1, RP_CTHREADS);
        if (q == 0 && blk < nblk) {
            double v[6] = {0, 0, 0, 0, 0, 0};
            double mx = 0.0;
            if (j < n) {
                double sum = 0.0;
#pragma unroll
                for (int k = 0; k < 8; ++k) sum += csh[grp][k][lane];
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
                mx = atw;
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = warp_sum(v[k]);
            mx = warp_max(mx);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) a.gf_part[(size_t)blk * 8 + k] = v[k];
                a.gf_part[(size_t)blk * 8 + 6] = mx;
            }
        }
        named_bar_sync(1, RP_CTHREADS);   // csh is free again
    }
    named_bar_sync(1, RP_CTHREADS);
    if (tid == 0) {
        __threadfence();
        glast = atomicAdd(a.bar + 2, 1u) == (unsigned)(G - 1) ? 1 : 0;
    }
    named_bar_sync(1, RP_CTHREADS);
    if (!glast) return;
    __threadfence();
    unsigned long long tm[4];
    if (a.timed && tid == 0) tm[0] = gtimer();
    __shared__ double gsh[8][8];
    double acc[6] = {0, 0, 0, 0, 0, 0}, am = -1e300, ls = 0.0;
    if (tid < 256) {
        for (int bb = tid; bb < nblk; bb += 256) {
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] += __ldcg(a.gf_part + (size_t)bb * 8 + k);
            am = fmax(am, __ldcg(a.gf_part + (size_t)bb * 8 + 6));
        }
        for (int bb = tid; bb < G; bb += 256) ls += __ldcg(a.rg.loss_part + bb);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = warp_sum(acc[k]);
    am = warp_max(am);
    ls = warp_sum(ls);
    if (lane == 0 && wid < 8) {
#pragma unroll
        for (int k = 0; k < 6; ++k) gsh[k][wid] = acc[k];
        gsh[6][wid] = am;
        gsh[7][wid] = ls;
    }
    named_bar_sync(1, RP_CTHREADS);
    double o[8];
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = warp_sum(lane < 8 ? gsh[k][lane] : 0.0);
        o[6] = warp_max(lane < 8 ? gsh[6][lane] : -1e300);
        o[7] = warp_sum(lane < 8 ? gsh[7][lane] : 0.0);
    }
    // the loop's decisions on a shared copy of the state's head (the slice buffer is free here)
    static_assert(sizeof(VT) * CGL_SLICE_MAX >= kStateHeadBytes, "slice buffer too small for the state head");
    DevState* S = a.S;
    if (a.timed && tid == 0) tm[1] = gtimer();
    loop_decide_shared(
        S, reinterpret_cast<unsigned long long*>(sh.vsl), tid, RP_CTHREADS, [] { named_bar_sync(1, RP_CTHREADS); },
        [&](DevState* Ss) {   // the totals, into the copy and the state
            for (DevState* T : {Ss, S}) {
                T->rd2 = o[0];
                T->rhou2 = o[1];
                T->g2 = o[2];
                T->excess2 = o[3];
                T->gx1 = o[4];
                T->gx2 = o[5];
                T->atw_inf = o[6];
                T->loss_sum = o[7];
            }
        },
        [&](DevLoop* Lc, DevState* Ss) {
            loop_phase_a(Lc, Ss);
            if (Lc->skip_kkt) loop_phase_b(Lc, Ss, kpow_next);
            if (a.timed) tm[2] = gtimer();
            if (a.use_cond) {
                cudaGraphSetConditional((cudaGraphConditionalHandle)a.kkt_cond, Lc->skip_kkt ? 0u : 1u);
                if (Lc->skip_kkt) cudaGraphSetConditional((cudaGraphConditionalHandle)a.loop_cond, Lc->cont ? 1u : 0u);
            }
        });
    if (a.timed && tid == 0) {   // the launch's last work: its span, and the start of the next gap
        const unsigned long long t = gtimer();
        const unsigned long long f0 = __ldcg(&S->cgl_fin0);
        S->cgl_tail_ns[0] += tm[0] > f0 ? (double)(tm[0] - f0) : 0.0;
        S->cgl_tail_ns[1] += (double)(tm[1] - tm[0]);
        S->cgl_tail_ns[2] += (double)(tm[2] - tm[1]);
        S->cgl_tail_ns[3] += (double)(t - tm[2]);
        S->cgl_span_ns += (double)(t - S->cgl_t0);
        S->cgl_last_end = t;
    }
}

// CTA 0, thread 0 of a timed launch: adds the time since the last mark to phase k
template <typename VT>
GENIOS_DEV void phase_mark(const CgLoopArgs& a, CglShared<VT>& sh, int k) {
    if (a.timed && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t = gtimer();
        a.S->cgl_phase_ns[k] += (double)(t - sh.t_mark);
        sh.t_mark = t;
    }
}

// The fused gradient pass of one CTA (a.grad): stages of the CTA's rows from the ring at
// v = x, the partial row of A^T l'(A x - b) and the CTA's loss sum.  Sets the producer's stop
// flag once the pass has taken its stages; false (the same in every consumer thread) on a wait
// that ran out.
template <int P, int NCH>
GENIOS_DEV bool fused_grad_pass(const CgLoopArgs& a, CglShared<typename VType<P>::T>& sh,
                                             unsigned char* smem, uint64_t* full, uint64_t* empty, int rps,
                                             int nst_cap, int& cs, int& par) {
    using AS = AStore<P>;
    constexpr int VEC = AS::VEC;
    using VT = typename VType<P>::T;
    const RowpassArgs& rp = a.rp;
    const int tid = threadIdx.x, lane = tid & 31, b = blockIdx.x;
    const int64_t row_bytes = rp.lda * (int64_t)sizeof(typename AS::T);
    const int64_t stage_bytes = (int64_t)rps * row_bytes;
    const int nchunk_row = (int)(row_bytes / 16);
    const int64_t n = rp.n;
    const VT* xg = static_cast<const VT*>(a.zu_x);
    VT vr[NCH][VEC], yr[NCH][VEC];
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = tid + k * RP_CTHREADS;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int64_t j = (int64_t)c * VEC + e;
            vr[k][e] = (c < nchunk_row && j < n && GCHK(rp.dbg, j, n)) ? __ldcg(xg + j) : VT(0);
            yr[k][e] = VT(0);
        }
    }
    double lsum = 0.0;
    VT wt_unused = VT(0);
    const int nstage_work = sh.nstage_work;
    const int64_t r0 = sh.r0, nrows = sh.nrows;
    VT* red = reinterpret_cast<VT*>(empty + nst_cap);
    bool ok = true;
    for (int w = 0; w < nstage_work; ++w, ++cs) {
        const int s = cs % nst_cap;
        const int use = cs / nst_cap;
        const bool got = mbar_wait_bounded(&full[s], (uint32_t)(use & 1), rp.wait_limit);
        if (named_bar_or(2, RP_CTHREADS, !got)) {
            if (tid == 0) atomicCAS(reinterpret_cast<int*>(&a.S->cg_fault), 0, DERR_TIMEOUT_FULL);
            ok = false;
            break;
        }
        rp_consume_stage<P, NCH, RP_GRAD>(a.rg, smem, smem + (size_t)s * stage_bytes,
                                          (int)min((int64_t)rps, nrows - (int64_t)w * rps), r0 + (int64_t)w * rps,
                                          row_bytes, nchunk_row, rps, red, par, vr, yr, lsum, false, wt_unused);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (tid == 0) *reinterpret_cast<volatile int32_t*>(&sh.stop) = 1;
    if (!ok) return false;
    VT* Pout = static_cast<VT*>(rp.partial) + (int64_t)b * rp.ldp;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = tid + k * RP_CTHREADS;
        if (c < nchunk_row) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int64_t j = (int64_t)c * VEC + e;
                if (j < rp.ldp && GCHK(rp.dbg, (long long)b * rp.ldp + j, rp.partial_len)) Pout[j] = yr[k][e];
            }
        }
    }
    // the rows' loss values sit in the lsum of one lane per row: a fixed-order CTA sum
    const double ls = csum(lsum, sh.dsh16);
    if (tid == 0) a.rg.loss_part[b] = ls;
    return true;
}

// Thread 0 of each CTA, before the x-step: its parameters (from the device-side loop's state when
// there is one) and a fresh CG state.
template <typename VT>
GENIOS_DEV void xstep_begin(const CgLoopArgs& a, CglShared<VT>& sh) {
    if (a.loop != nullptr) {
        const DevLoop* L = a.loop;
        sh.rho = __ldcg(&L->rho);
        sh.u_scale = __ldcg(&L->u_scale);
        sh.nu = __ldcg(&L->nu);
        sh.tol = __ldcg(&L->tol);
        sh.zu_rho = sh.rho;
        sh.zu_lam1 = __ldcg(&L->lam1);
        if (blockIdx.x == 0) a.loop->last_cg = __ldcg(&L->k);
    } else {
        sh.rho = a.rho;
        sh.u_scale = a.u_scale;
        sh.nu = a.nu;
        sh.tol = a.tol;
        sh.zu_rho = a.zu_rho;
        sh.zu_lam1 = a.zu_lam1;
    }
    sh.it = 0;
    sh.start = 1;
    sh.rz_old = sh.rhs2 = sh.rr = sh.rz = sh.alpha = sh.beta = sh.pq = VT(0);
}

template <int P, int NCH>
__global__ void __launch_bounds__(RP_THREADS, 1) cgloop_kernel(const CgLoopArgs a, const int rps, const int nst_cap) {
    using AS = AStore<P>;
    constexpr int VEC = AS::VEC;
    using VT = typename VType<P>::T;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ CglShared<VT> sh;

    const RowpassArgs& rp = a.rp;
    DevState* S = a.S;
    const int tid = threadIdx.x;
    const int G = gridDim.x, b = blockIdx.x;
    const int64_t row_bytes = rp.lda * (int64_t)sizeof(typename AS::T);
    const int64_t stage_bytes = (int64_t)rps * row_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nst_cap * stage_bytes);
    uint64_t* empty = full + nst_cap;

    // graph-form loop: the WHILE condition is cleared here and set again by the iteration's
    // last finishing kernel when the loop is to go on
    if (a.use_cond && b == 0 && tid == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)a.loop_cond, 0u);
    // device-side ADMM loop: nothing to do once the solve has stopped (the flag was written by an
    // earlier kernel in the stream, so every CTA reads the same value)
    if (a.loop != nullptr && a.loop->stop != 0) return;
    if (tid == 0) {
        xstep_begin<VT>(a, sh);
        for (int s = 0; s < nst_cap; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], RP_CWARPS);
        }
        fence_mbar_init();
        const int64_t r0 = (rp.m * (int64_t)b) / G, r1 = (rp.m * ((int64_t)b + 1)) / G;
        sh.r0 = r0;
        sh.nrows = r1 - r0;
        sh.nstage_work = (int)((r1 - r0 + rps - 1) / rps);
        const int64_t j0 = rp.n * b / G, j1 = rp.n * (b + 1) / G;
        sh.j0 = j0;
        sh.ns = (int)(j1 - j0);
        sh.epoch = 0;
        sh.stop = 0;
        sh.t_start = 0ull;
        if (a.timed && b == 0) {   // before this CTA's first arrival: no H phase has begun
            sh.t_start = gtimer();
            sh.t_mark = sh.t_start;
            S->hv_t0 = ~0ull;
            S->hv_t1 = 0ull;
            S->cgl_t0 = sh.t_start;
            const unsigned long long prev = S->cgl_last_end;
            if (prev != 0ull && sh.t_start > prev) S->cgl_gap_ns += (double)(sh.t_start - prev);
        }
    }
    for (int i = tid; i < 128; i += RP_THREADS) sh.lamsh[i] = i < a.sk ? (VT)a.lam[i] : VT(0);
    __syncthreads();

    // ------------------------------------------------------------------ producer warp
    if (tid >= RP_CTHREADS) {
        const int nstage_work = sh.nstage_work;
        if (tid == RP_CTHREADS && nstage_work > 0) {
            const char* Ab = static_cast<const char*>(rp.A);
            const uint64_t pol = l2_evict_first_policy();
            const int64_t r0 = sh.r0, nrows = sh.nrows;
            volatile int32_t* stop = &sh.stop;
            long long issued = 0;
            for (long long st = 0;; ++st) {
                const int s = (int)(st % nst_cap);
                const long long use = st / nst_cap;
                if (use > 0) {   // slot free, or the consumers have stopped
                    const uint32_t par = (uint32_t)((use - 1) & 1);
                    bool got = mbar_try_wait(&empty[s], par);
                    const long long t0 = clock64();
                    while (!got && *stop == 0) {
                        if (clock64() - t0 > rp.wait_limit) {
                            atomicCAS(reinterpret_cast<int*>(&S->cg_fault), 0, DERR_TIMEOUT_EMPTY);
                            break;
                        }
                        got = mbar_try_wait(&empty[s], par);
                    }
                    if (!got) break;
                }
                if (*stop != 0) break;
                const int ws = (int)(st % nstage_work);   // stage of the pass
                const int64_t rows = min((int64_t)rps, nrows - (int64_t)ws * rps);
                const uint32_t bytes = (uint32_t)(rows * row_bytes);
                const int64_t off = (r0 + (int64_t)ws * rps) * row_bytes;
#ifdef GENIOS_CHECKED
                if (!GCHK(rp.dbg, (long long)s * stage_bytes + (long long)bytes - 1, (long long)nst_cap * stage_bytes) ||
                    !GCHK(rp.dbg, r0 + (long long)ws * rps + rows - 1, rp.m)) break;
#endif
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s_hint(smem + (size_t)s * stage_bytes, Ab + off, bytes, &full[s], pol);
                issued = st + 1;
            }
            // every copy issued must land before the CTA's shared memory is released
            for (long long st = std::max(0LL, issued - nst_cap); st < issued; ++st)
                mbar_wait_bounded(&full[st % nst_cap], (uint32_t)((st / nst_cap) & 1), drain_limit(rp.wait_limit));
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int lane = tid & 31;
    cg_start<VT>(a, sh);
    bool ok = grid_sync(a, sh);   // false once a wait ran out here or in another CTA
    int cs = 0, par = 0;   // stages consumed (the ring position), row-total scratch half
    while (ok && cg_direction<VT>(a, sh)) {
        phase_mark(a, sh, 4);
        if (!(ok = grid_sync(a, sh))) break;
        phase_mark(a, sh, 5);

        // ---- H: y_b = A_b^T diag(d_b) A_b p
        if (a.timed && tid == 0) atomicMin(&S->hv_t0, gtimer());
        const int nchunk_row = (int)(row_bytes / 16);
        const int64_t n = rp.n;
        const VT* p = static_cast<const VT*>(a.p);
        VT vr[NCH][VEC], yr[NCH][VEC];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const int c = tid + k * RP_CTHREADS;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int64_t j = (int64_t)c * VEC + e;
                vr[k][e] = (c < nchunk_row && j < n && GCHK(rp.dbg, j, n)) ? __ldcg(p + j) : VT(0);
                yr[k][e] = VT(0);
            }
        }
        double lsum_unused = 0.0;
        VT wt_unused = VT(0);
        const int nstage_work = sh.nstage_work;
        const int64_t r0 = sh.r0, nrows = sh.nrows;
        VT* red = reinterpret_cast<VT*>(empty + nst_cap);   // [2][RB][RP_CWARPS]
        bool hfault = false;
        for (int w = 0; w < nstage_work; ++w, ++cs) {
            const int s = cs % nst_cap;
            const int use = cs / nst_cap;
            const bool got = mbar_wait_bounded(&full[s], (uint32_t)(use & 1), rp.wait_limit);
            if (named_bar_or(2, RP_CTHREADS, !got)) {
                if (tid == 0) atomicCAS(reinterpret_cast<int*>(&S->cg_fault), 0, DERR_TIMEOUT_FULL);
                hfault = true;
                break;
            }
            rp_consume_stage<P, NCH, RP_HV>(rp, smem, smem + (size_t)s * stage_bytes,
                                            (int)min((int64_t)rps, nrows - (int64_t)w * rps), r0 + (int64_t)w * rps,
                                            row_bytes, nchunk_row, rps, red, par, vr, yr, lsum_unused, false, wt_unused);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (hfault) {
            ok = false;
            break;
        }
        {   // the partial y_b, and p^T y_b (summed over the CTAs: p^T A^T diag(d) A p)
            VT* Pout = static_cast<VT*>(rp.partial) + (int64_t)b * rp.ldp;
            VT py = VT(0);
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int c = tid + k * RP_CTHREADS;
                if (c < nchunk_row) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const int64_t j = (int64_t)c * VEC + e;
                        if (j < rp.ldp && GCHK(rp.dbg, (long long)b * rp.ldp + j, rp.partial_len)) Pout[j] = yr[k][e];
                        py = fma(vr[k][e], yr[k][e], py);
                    }
                }
            }
            py = csum(py, sh.sh16);
            if (tid == 0) static_cast<VT*>(a.part)[(size_t)G * CGL_ST + b] = py;
        }
        if (a.timed) {
            named_bar_sync(1, RP_CTHREADS);
            if (tid == 0) atomicMax(&S->hv_t1, gtimer());
        }
        phase_mark(a, sh, 0);
        if (!(ok = grid_sync(a, sh))) break;
        phase_mark(a, sh, 1);
        if (a.timed && b == 0 && tid == 0) {
            const unsigned long long t0 = S->hv_t0, t1 = S->hv_t1;
            if (t1 > t0) {
                S->hv_ns += (double)(t1 - t0);
                S->hv_count += 1;
            }
            S->hv_t0 = ~0ull;
            S->hv_t1 = 0ull;
        }

        // ---- Q
        if (!cg_step<VT>(a, sh)) break;
        phase_mark(a, sh, 2);
        if (!(ok = grid_sync(a, sh))) break;
        phase_mark(a, sh, 3);
    }

    // ---- the result is in delta; the producer stops here unless the gradient pass follows
    // (a.loop->halt was written by an earlier kernel: every CTA reads the same value)
    // (only the FP64 and FP32 instantiations carry the gradient pass: the quantised Hessian
    // streams of BF16 and FP8 are not the gradient's matrix, and leaving it out keeps their
    // register allocation as it was)
    constexpr bool kGradCapable = (P == P_FP32 || P == P_FP64);
    const bool gradp = kGradCapable && ok && a.grad && a.zu && a.loop != nullptr && a.loop->halt == 0;
    if (!gradp && tid == 0) *reinterpret_cast<volatile int32_t*>(&sh.stop) = 1;
    if (ok && a.zu) zu_phase<VT>(a, sh);
    // one thread records the final scalars
    if (b == 0 && tid == 0) {
        S->cg_it = sh.it;
        S->cg_done = 1;
        S->cg_guard = 0;
        S->rr = sh.rr;
        S->rz = sh.rz;
        S->rhs2 = sh.rhs2;
        S->pq = sh.pq;
        S->alpha = sh.alpha;
        S->beta = sh.beta;
        S->nu = sh.nu;
        S->tol = sh.tol;
        S->cg_max = a.cg_max;
        if (a.timed) S->cgl_iters += sh.it;
    }

    // ---- gradient pass at the new x over the CTA's rows (the ring already holds its first
    // stages), then its finish and the loop's decisions
    if (gradp) {
        phase_mark(a, sh, 4);   // the final stop test and the z/u update count as direction work
        if constexpr (kGradCapable) {
            bool gok = grid_sync(a, sh);   // x is complete in every slice
            if (gok) {
                gok = fused_grad_pass<P, NCH>(a, sh, smem, full, empty, rps, nst_cap, cs, par);
                if (gok) gok = grid_sync(a, sh);   // every partial row is written
            }
            phase_mark(a, sh, 6);
            if (a.timed && b == 0 && tid == 0) a.S->cgl_fin0 = gtimer();
            if (gok) grad_finish_phase<VT>(a, sh);
            phase_mark(a, sh, 7);
        }
    }
    if (tid == 0) *reinterpret_cast<volatile int32_t*>(&sh.stop) = 1;   // the producer leaves
    if (b == 0 && tid == 0 && a.timed) {
        S->cgl_ns += (double)(gtimer() - sh.t_start);
        S->cgl_count += 1;
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int P, int NCH>
static bool occupancy_ok(size_t smem) {
    auto kern = cgloop_kernel<P, NCH>;
    // the attribute bounds every launch of this instantiation, whatever shape planned it last
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CGL_SMEM_BUDGET) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, RP_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nb >= 1;
}

template <int P>
static bool occupancy_nch(int nch, size_t smem) {
    switch (nch) {
        case 1: return occupancy_ok<P, 1>(smem);
        case 2: return occupancy_ok<P, 2>(smem);
        case 3: return occupancy_ok<P, 3>(smem);
        case 4: return occupancy_ok<P, 4>(smem);
        case 6: return occupancy_ok<P, 6>(smem);
        case 8: return occupancy_ok<P, 8>(smem);
        case 10:
            if constexpr (P != P_FP64) return occupancy_ok<P, 10>(smem);
            else return false;
        default: return false;
    }
}

CgLoopPlan cgloop_plan(int prec, int64_t m, int64_t n, int64_t lda, int sk, size_t stage_target) {
    CgLoopPlan cp{};
    cp.ok = false;
    if (prec == P_HILO || sk < 0 || sk > 128) return cp;
    RowpassPlan p = rowpass_plan(prec, m, n, lda, CGL_SMEM_BUDGET, stage_target);
    if (!p.ok) return cp;
    const int sms = device_sm_count();
    if ((n + sms - 1) / sms > CGL_SLICE_MAX) return cp;
    bool ok = false;
    switch (prec) {
        case P_FP64: ok = occupancy_nch<P_FP64>(p.nch, p.smem); break;
        case P_FP32: ok = occupancy_nch<P_FP32>(p.nch, p.smem); break;
        case P_BF16: ok = occupancy_nch<P_BF16>(p.nch, p.smem); break;
        case P_FP8:  ok = occupancy_nch<P_FP8>(p.nch, p.smem); break;
        default: ok = false;
    }
    if (!ok) return cp;
    p.grid = sms;   // one CTA per SM; CTAs without rows still own a slice of the vectors
    cp.rp = p;
    cp.ok = true;
    return cp;
}

size_t cgloop_part_elems(int grid) { return (size_t)grid * (CGL_ST + 2); }
size_t cgloop_zu_offset_bytes(int grid) { return ((size_t)grid * (CGL_ST + 2) * 8 + 255) & ~size_t(255); }
size_t cgloop_gf_offset_bytes(int grid) { return cgloop_zu_offset_bytes(grid) + (((size_t)grid * 6 * 8 + 255) & ~size_t(255)); }

template <int P, int NCH>
static cudaError_t launch_cgl(const CgLoopArgs& a, const RowpassPlan& p, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(p.grid);
    cfg.blockDim = dim3(RP_THREADS);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cgloop_kernel<P, NCH>, a, p.rows_per_stage, p.nstages);
}

template <int P>
static cudaError_t dispatch_cgl(const CgLoopArgs& a, const RowpassPlan& p, cudaStream_t s) {
    switch (p.nch) {
        case 1: return launch_cgl<P, 1>(a, p, s);
        case 2: return launch_cgl<P, 2>(a, p, s);
        case 3: return launch_cgl<P, 3>(a, p, s);
        case 4: return launch_cgl<P, 4>(a, p, s);
        case 6: return launch_cgl<P, 6>(a, p, s);
        case 8: return launch_cgl<P, 8>(a, p, s);
        case 10:
            if constexpr (P != P_FP64) return launch_cgl<P, 10>(a, p, s);
            else return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t cgloop_launch(const CgLoopPlan& pl, const CgLoopArgs& c, cudaStream_t s) {
    if (!pl.ok || c.sk > 128 || c.sk < 0 || c.bar == nullptr || c.part == nullptr) return cudaErrorInvalidValue;
    CgLoopArgs a = c;
    a.rp.mode = RP_HV;
    a.rp.smem_bytes = (long long)pl.rp.smem;
    a.rp.partial_len = (long long)pl.rp.grid * c.rp.ldp;
    a.rg.smem_bytes = a.rp.smem_bytes;
    a.rg.partial_len = a.rp.partial_len;
    if (c.grad && (c.loop == nullptr || !c.zu || c.g_out == nullptr || c.gf_part == nullptr ||
                   c.rg.b == nullptr || c.rg.loss_part == nullptr))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(c.bar, 0, 3 * sizeof(unsigned), s);   // grid barrier, last-CTA counts
    if (e != cudaSuccess) return e;
    switch (c.rp.prec) {
        case P_FP64: return dispatch_cgl<P_FP64>(a, pl.rp, s);
        case P_FP32: return dispatch_cgl<P_FP32>(a, pl.rp, s);
        case P_BF16: return dispatch_cgl<P_BF16>(a, pl.rp, s);
        case P_FP8:  return dispatch_cgl<P_FP8>(a, pl.rp, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace genios
