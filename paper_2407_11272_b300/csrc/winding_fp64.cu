// FP64 re-evaluation of the flagged queries (|w - 0.5| < 1e-3 or within 1e-3 of a triangle):
// the full sum of Eq. (5) over every face, each term ATAN2(N, D) of Eq. (7)/(8) in FP64, then
// w and the occupancy of those queries are overwritten. The flagged list and its length stay on
// the device; a persistent grid walks the list in batches of kRsQB queries, and each batch is
// reduced across the CTA in a fixed order (deterministic).
#include <math.h>

#include "dv_internal.cuh"

namespace dv {

constexpr int kReThreads = 256;
// The faces are visited in strip order (strips.cu): every thread walks a
// contiguous run of events and keeps, per query of the batch, the offset, |P - q| and the dot
// with the previous vertex of the two most recent vertices; a face then costs one FP64 square
// root and two dots instead of three of each (D and N as in the FP32 strip kernel). A thread's
// run starts with up to two warm-up events (vertex part only). The FP64 pipe bounds this
// kernel, not instruction issue, so the state is simply shifted after each event.
constexpr int kRsQB = 2;

struct Slot64 {
    double ax[kRsQB], ay[kRsQB], az[kRsQB], l[kRsQB], e[kRsQB];
};

// Sum of the half angles ATAN2(N, D) of Eq. (7)/(8) without an arctangent per face. For a face
// with D > 8|N| (seen under less than ~0.25 sr, almost every face) ATAN2(N, D) is the argument
// of z = D + iN, |arg z| < atan(1/8), and a sum of arguments is the argument of the product of
// the z, counted with its turns: the running product P of a thread's fast faces changes its
// argument by less than 0.125 rad per factor, so it passes the negative real axis exactly when
// Im P changes sign while Re P < 0, upwards (+1 turn) when Im P goes from >= +0 to <= -0 and
// downwards otherwise (sign bits, matching atan2's +-pi on that axis). At the end
// sum = ATAN2(Im P, Re P) + 2 pi turns. Each factor is scaled by the power of two that brings D
// into [1, 2) (exact), so |P| only grows, by less than 2.01 per factor, and P is rescaled by a
// power of two every kRenorm faces. Per fast face this costs a complex product instead of a
// division and a polynomial; every other face (D <= 8|N|) adds ATAN2 with Eq. (8)'s
// conventions: -0 -> +0, ATAN2(0, 0) = 0, and 0 for a query on one of the face's vertices
// (a distance of exactly 0, where N and D vanish).
constexpr int kRenorm = 64;

__device__ __forceinline__ double slow_half_angle64(double N, double D, double lV, double l1, double l2) {
    if (lV == 0.0 || l1 == 0.0 || l2 == 0.0) return 0.0;
    if (N == 0.0 && D == 0.0) return 0.0;
    return atan2(N + 0.0, D);
}

// 2^-e for x in [2^e, 2^(e+1)), built from x's exponent field (x > 0; clamped to normal scales).
__device__ __forceinline__ double inv_pow2_of(double x) {
    const int e = (__double2hiint(x) >> 20) & 0x7ff;
    int f = 2046 - e;
    f = f < 1 ? 1 : (f > 2046 ? 2046 : f);
    return __hiloint2double(f << 20, 0);
}

struct ArgProduct {
    double re, im;
    int turns;
};

__device__ __forceinline__ void arg_product_mul(ArgProduct &P, double D, double N) {
    const double sc = inv_pow2_of(D);
    const double dr = D * sc, di = N * sc;
    const double nr = fma(P.re, dr, -P.im * di);
    const double ni = fma(P.re, di, P.im * dr);
    const bool so = __double2hiint(P.im) < 0, sn = __double2hiint(ni) < 0;
    if (so != sn && nr < 0.0) P.turns += so ? -1 : 1;
    P.re = nr;
    P.im = ni;
}

__global__ void __launch_bounds__(kReThreads, 2)
    reeval_strip_kernel(const StripRec64 *__restrict__ srec, int64_t ne, GridD g, const float *__restrict__ queries,
                        const int *__restrict__ list, const int *__restrict__ count, int64_t nq, float *w_out,
                        uint8_t *occ_out, unsigned *maxdiff_bits, int *occ_changed) {
    __shared__ double red[kReThreads / 32][kRsQB];
    const int M = *count;
    const int nb = (M + kRsQB - 1) / kRsQB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunk = (ne + kReThreads - 1) / kReThreads;
    const int64_t eb = (int64_t)threadIdx.x * chunk;
    const int64_t ee = eb + chunk < ne ? eb + chunk : ne;
    const int64_t es = eb < 2 ? 0 : eb - 2;  // warm-up start
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        double qx[kRsQB], qy[kRsQB], qz[kRsQB], sum[kRsQB];
        ArgProduct prod[kRsQB];
        int ids[kRsQB];
#pragma unroll
        for (int j = 0; j < kRsQB; ++j) {
            const int k = b * kRsQB + j < M ? b * kRsQB + j : M - 1;
            const int idx = DV_INB(k, nq, kSiteReevalQuery) && DV_INB(list[k], nq, kSiteReevalQuery) ? list[k] : 0;
            ids[j] = idx;
            if (queries) {
                qx[j] = (double)queries[3 * (int64_t)idx];
                qy[j] = (double)queries[3 * (int64_t)idx + 1];
                qz[j] = (double)queries[3 * (int64_t)idx + 2];
            } else {
                const int ix = idx % g.n[0], iy = (idx / g.n[0]) % g.n[1], iz = idx / (g.n[0] * g.n[1]);
                qx[j] = g.lo[0] + ((double)ix + 0.5) * g.h[0];
                qy[j] = g.lo[1] + ((double)iy + 0.5) * g.h[1];
                qz[j] = g.lo[2] + ((double)iz + 0.5) * g.h[2];
            }
            sum[j] = 0.0;
            prod[j] = ArgProduct{1.0, 0.0, 0};
        }
        int nfac = 0;
        Slot64 P1, P2;
#pragma unroll
        for (int j = 0; j < kRsQB; ++j) {
            P1.ax[j] = P1.ay[j] = P1.az[j] = P1.l[j] = P1.e[j] = 0.0;
            P2.ax[j] = P2.ay[j] = P2.az[j] = P2.l[j] = P2.e[j] = 0.0;
        }
        for (int64_t ev = es; ev < ee; ++ev) {
            if (!DV_INB(ev, ne, kSiteReevalEvent)) break;
            const StripRec64 r = srec[ev];
            const bool face = r.flag != 0.0 && ev >= eb;
            Slot64 V;
#pragma unroll
            for (int j = 0; j < kRsQB; ++j) {
                V.ax[j] = r.v[0] - qx[j];
                V.ay[j] = r.v[1] - qy[j];
                V.az[j] = r.v[2] - qz[j];
                V.l[j] = sqrt(V.ax[j] * V.ax[j] + V.ay[j] * V.ay[j] + V.az[j] * V.az[j]);
                V.e[j] = V.ax[j] * P1.ax[j] + V.ay[j] * P1.ay[j] + V.az[j] * P1.az[j];
            }
            if (face) {
#pragma unroll
                for (int j = 0; j < kRsQB; ++j) {
                    const double d2 = V.ax[j] * P2.ax[j] + V.ay[j] * P2.ay[j] + V.az[j] * P2.az[j];
                    const double N = V.ax[j] * r.n[0] + V.ay[j] * r.n[1] + V.az[j] * r.n[2];
                    const double D = (V.l[j] * P1.l[j] + V.e[j]) * P2.l[j] + V.l[j] * P1.e[j] + P1.l[j] * d2;
                    if (D > 8.0 * fabs(N))
                        arg_product_mul(prod[j], D, N);
                    else
                        sum[j] += slow_half_angle64(N, D, V.l[j], P1.l[j], P2.l[j]);
                }
                if (++nfac == kRenorm) {
#pragma unroll
                    for (int j = 0; j < kRsQB; ++j) {
                        const double sc = inv_pow2_of(fmax(fabs(prod[j].re), fabs(prod[j].im)));
                        prod[j].re *= sc;
                        prod[j].im *= sc;
                    }
                    nfac = 0;
                }
            }
            P2 = P1;
            P1 = V;
        }
#pragma unroll
        for (int j = 0; j < kRsQB; ++j) {
            double v = sum[j] + (atan2(prod[j].im, prod[j].re) + kTwoPiD * prod[j].turns);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
            if (lane == 0) red[warp][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < kRsQB && b * kRsQB + (int)threadIdx.x < M) {
            const int j = threadIdx.x;
            double t = 0.0;
            for (int w = 0; w < kReThreads / 32; ++w) t += red[w][j];
            const double w64 = t * kInv2PiD;
            const int idx = ids[j];
            const float w32 = w_out[idx];
            const float wn = (float)w64;
            w_out[idx] = wn;
            const uint8_t o_new = w64 > 0.5 ? 1 : 0;
            if (occ_out) occ_out[idx] = o_new;
            const float diff = fabsf(w32 - wn);
            atomicMax(maxdiff_bits, __float_as_uint(isfinite(diff) ? diff : 3.0e38f));
            if ((w32 > 0.5f ? 1 : 0) != o_new) atomicAdd(occ_changed, 1);
        }
        __syncthreads();
    }
}

cudaError_t launch_reeval_fp64(const StripRec64 *srec64, int64_t ne, const GridD *g, const float *queries,
                               const int *flag_list, const int *flag_count, int64_t max_flagged, float *w_out,
                               uint8_t *occ_out, unsigned *stat_maxdiff_bits, int *stat_occ_changed, int num_sms,
                               cudaStream_t s) {
    if (!srec64 || ne < 1) return cudaErrorInvalidValue;
    GridD gd{};
    if (g) gd = *g;
    int64_t blocks = 4LL * num_sms;
    const int64_t need = (max_flagged + kRsQB - 1) / kRsQB;
    if (need < blocks) blocks = need > 0 ? need : 1;
    prof_begin("reeval_fp64", s);
    reeval_strip_kernel<<<(unsigned)blocks, kReThreads, 0, s>>>(srec64, ne, gd, queries, flag_list, flag_count,
                                                                max_flagged, w_out, occ_out, stat_maxdiff_bits,
                                                                stat_occ_changed);
    count_launch();
    prof_end("reeval_fp64", s);
    return cudaGetLastError();
}

}  // namespace dv
