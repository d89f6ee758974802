// The consumer side of the fused rowpass (rowpass.cu), shared with the persistent CG kernel
// (cgloop.cu): one stage of whole rows in shared memory -> row dot products t_i = a_i^T v,
// row weights w_i, and y += w_i a_i on the thread's column slice.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace genios {

constexpr int RP_CWARPS = 16;
constexpr int RP_CTHREADS = RP_CWARPS * 32;
constexpr int RP_THREADS = RP_CTHREADS + 32;

// rows per barrier group: 8 held 16-byte chunks per thread, halved for the FP8 and split-BF16
// streams whose chunks expand to 16 / 2 x 8 values (register pressure)
__host__ __device__ constexpr int rp_rb(int prec, int nch) {
    return (nch >= 8 ? 1 : (8 / nch)) / ((prec == P_FP8 || prec == P_HILO) && nch < 8 ? 2 : 1) > 0
               ? (nch >= 8 ? 1 : (8 / nch)) / ((prec == P_FP8 || prec == P_HILO) && nch < 8 ? 2 : 1)
               : 1;
}

// Consumes `rows` rows (global indices i0, i0 + 1, ...) of one stage at sb.  Called by the
// 512 consumer threads together (it synchronises them with named barrier 1).  red: the
// [2][RB][RP_CWARPS] row-total scratch; par alternates its halves.  vr / yr: the thread's
// chunks of v and of the partial y.  Gradient mode adds each row's loss value into the lsum of
// one consumer thread (the caller sums the threads' lsum in a fixed order);
// Hv mode with want_wt adds sum_i w_i t_i (the rows' share of v^T A^T diag(d) A v) into wt
// (thread 0).
template <int P, int NCH, int MODE>
GENIOS_DEV void rp_consume_stage(const RowpassArgs& a, const unsigned char* smem, const unsigned char* sb,
                                 const int rows, const int64_t i0, const int64_t row_bytes, const int nchunk_row,
                                 const int rps, typename VType<P>::T* red, int& par,
                                 typename VType<P>::T (&vr)[NCH][AStore<P>::VEC],
                                 typename VType<P>::T (&yr)[NCH][AStore<P>::VEC], double& lsum,
                                 const bool want_wt, typename VType<P>::T& wt) {
    using AS = AStore<P>;
    constexpr int VEC = AS::VEC;
    using VT = typename VType<P>::T;
    constexpr bool HILO = (P == P_HILO);
    constexpr bool FP8 = (P == P_FP8);
    constexpr int RB = rp_rb(P, NCH);
    // the row group's chunks are held in registers between the dot and the update only while
    // v, y and the held chunks fit in about 64 of the 96 registers a thread has (17 warps per
    // CTA); wider rows re-read them from shared memory instead of spilling
    constexpr bool HOLD = (NCH * RB <= 8) && (2 * NCH * VEC * (int)(sizeof(VT) / 4) + 4 * NCH * RB <= 64);
    constexpr bool PK = sizeof(VT) == 4 && !HILO;   // float32 lanes: packed f32x2 FMAs
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const VT* dvec = static_cast<const VT*>(a.d);
    const VT* bvec = static_cast<const VT*>(a.b);
    VT* Wout = static_cast<VT*>(a.W_out);
    VT* Dout = static_cast<VT*>(a.D_out);
    for (int rr = 0; rr < rows; rr += RB) {
        uint4 hold[HOLD ? RB : 1][HOLD ? NCH : 1];
        uint4 holdlo[(HOLD && HILO) ? RB : 1][(HOLD && HILO) ? NCH : 1];
        VT dot[RB];
        uint64_t dot2[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            dot[q] = VT(0);
            dot2[q] = 0ull;   // +0.0f, +0.0f
            if (rr + q < rows) {
                const unsigned char* rowp = sb + (size_t)(rr + q) * row_bytes;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int c = tid + k * RP_CTHREADS;
                    if (c < nchunk_row &&
                        GCHK(a.dbg, (rowp - smem) + (long long)c * 16 + (HILO ? (long long)rps * row_bytes : 0) + 15, a.smem_bytes)) {
                        const uint4 raw = ld_shared_v4(rowp + (size_t)c * 16);
                        VT f[VEC];
                        decode_chunk(raw, f);
                        if constexpr (HILO) {
                            const uint4 rl = ld_shared_v4(rowp + (size_t)rps * row_bytes + (size_t)c * 16);
                            VT g[VEC];
                            decode_chunk(rl, g);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) f[e] += g[e];
                            if constexpr (HOLD) holdlo[q][k] = rl;
                        }
                        if constexpr (HOLD) hold[q][k] = raw;
                        if constexpr (PK) {
#pragma unroll
                            for (int e = 0; e < VEC; e += 2)
                                dot2[q] = fma2(f2pack(f[e], f[e + 1]), f2pack(vr[k][e], vr[k][e + 1]), dot2[q]);
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e) dot[q] = fma(f[e], vr[k][e], dot[q]);
                        }
                    }
                }
            }
            if constexpr (PK) {
                const float2 d2 = f2unpack(dot2[q]);
                dot[q] = d2.x + d2.y;
            }
        }
        // Row totals of the RB dot products.  Within the warp a transposed reduce-scatter:
        // each halving step sends half of a lane's values across and keeps the other half,
        // so after log2(RB) steps lane group g = lane / GS (GS = 32 / RB lanes) holds row g's
        // partial, finished over the group (RB - 1 + log2(GS) shuffles instead of 5 RB).
        // Across the 16 warps, group g folds row g's 16 warp partials the same way and the
        // totals are broadcast from the groups.
        constexpr int LR = RB == 1 ? 0 : RB == 2 ? 1 : RB == 4 ? 2 : 3;
        static_assert((1 << LR) == RB, "rows per barrier group must be 1, 2, 4 or 8");
        constexpr int GS = 32 >> LR;
        {
#pragma unroll
            for (int l = 0; l < LR; ++l) {
                const int off = 16 >> l;
                const bool up = (lane & off) != 0;
                const int half = RB >> (l + 1);
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const VT keep = up ? dot[i + half] : dot[i];
                    const VT send = up ? dot[i] : dot[i + half];
                    dot[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
#pragma unroll
            for (int off = GS >> 1; off > 0; off >>= 1) dot[0] += __shfl_xor_sync(0xffffffffu, dot[0], off);
            if ((lane & (GS - 1)) == 0 &&
                GCHK(a.dbg, (long long)(reinterpret_cast<unsigned char*>(red + (par * RB + lane / GS) * RP_CWARPS + wid) - smem) + (long long)sizeof(VT) - 1, a.smem_bytes))
                red[(par * RB + lane / GS) * RP_CWARPS + wid] = dot[0];
        }
        named_bar_sync(1, RP_CTHREADS);
        VT wq[RB];
        {
            const int g = lane / GS, sidx = lane & (GS - 1);
            VT t = VT(0);
#pragma unroll
            for (int w = sidx; w < RP_CWARPS; w += GS) t += red[(par * RB + g) * RP_CWARPS + w];
#pragma unroll
            for (int off = GS >> 1; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if constexpr (MODE == RP_HV) {
                VT tot[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) tot[q] = __shfl_sync(0xffffffffu, t, q * GS);
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    VT tq = tot[q];
                    wq[q] = VT(0);
                    if (rr + q < rows) {
                        const int64_t i = i0 + rr + q;
                        VT sc = VT(1);
                        if constexpr (FP8) sc = GCHK(a.dbg, i, a.m) ? (VT)__ldg(a.row_scale + i) : VT(1);
                        tq *= sc;
                        VT w = (dvec != nullptr && GCHK(a.dbg, i, a.m)) ? dvec[i] * tq : tq;
                        wq[q] = w * sc;
                        if (want_wt && tid == 0) wt += w * tq;
                    }
                }
            } else {
                // Row g's weight l'(t_g - b_g) is formed by its own lane group (one loss
                // derivative per lane instead of RB per thread), then broadcast.  The row's loss
                // value and l'' are formed by one lane, in a warp that rotates with the row, and
                // go to W_out / D_out and to that lane's share of the loss sum.
                VT w = VT(0);
                const int64_t i = i0 + rr + g;
                if (rr + g < rows && GCHK(a.dbg, i, a.m)) {
                    VT sc = VT(1);
                    if constexpr (FP8) sc = (VT)__ldg(a.row_scale + i);
                    const VT u = t * sc - bvec[i];
                    w = loss_d1<VT>(a.loss, u) * sc;
                    if (sidx == 0 && wid == (int)(i % RP_CWARPS)) {
                        VT l0, l1, l2;
                        loss_eval<VT>(a.loss, u, l0, l1, l2);
                        if (Wout) Wout[i] = l1;
                        if (Dout) Dout[i] = l2;
                        lsum += (double)l0;
                    }
                }
#pragma unroll
                for (int q = 0; q < RB; ++q) wq[q] = __shfl_sync(0xffffffffu, w, q * GS);
            }
        }
        par ^= 1;
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            if (rr + q < rows) {
                const unsigned char* rowp = sb + (size_t)(rr + q) * row_bytes;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int c = tid + k * RP_CTHREADS;
                    if (c < nchunk_row &&
                        GCHK(a.dbg, (rowp - smem) + (long long)c * 16 + (HILO ? (long long)rps * row_bytes : 0) + 15, a.smem_bytes)) {
                        uint4 raw;
                        if constexpr (HOLD) raw = hold[q][k];
                        else raw = ld_shared_v4(rowp + (size_t)c * 16);
                        VT f[VEC];
                        decode_chunk(raw, f);
                        if constexpr (HILO) {
                            uint4 rl;
                            if constexpr (HOLD) rl = holdlo[q][k];
                            else rl = ld_shared_v4(rowp + (size_t)rps * row_bytes + (size_t)c * 16);
                            VT g[VEC];
                            decode_chunk(rl, g);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) f[e] += g[e];
                        }
                        if constexpr (PK) {
                            const uint64_t w2 = f2pack(wq[q], wq[q]);
#pragma unroll
                            for (int e = 0; e < VEC; e += 2) {
                                const float2 y2 = f2unpack(fma2(w2, f2pack(f[e], f[e + 1]),
                                                                f2pack(yr[k][e], yr[k][e + 1])));
                                yr[k][e] = y2.x;
                                yr[k][e + 1] = y2.y;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e) yr[k][e] = fma(wq[q], f[e], yr[k][e]);
                        }
                    }
                }
            }
        }
    }
}

}  // namespace genios
