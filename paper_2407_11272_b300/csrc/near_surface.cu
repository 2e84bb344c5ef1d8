// Near-surface selection for the FP64 re-evaluation: flag every query within kNearDist of a
// triangle (Euclidean distance, conservative: a small FP32 margin only adds queries).
//
// Grid path: a warp per (face, z-slice group) visits the voxel centres inside the face's
// bounding box grown by the threshold, computes the point-triangle distance in FP32 and sets
// near_flag[q] = 1.
// Work is O(sum over faces of voxels in the grown box), far below the F x Q pair count.
// List path: queries binned into cells over the mesh's grown box; each face tests the queries
// of the cells its grown box overlaps.
#include <math.h>

#include "dv_internal.cuh"

namespace dv {

constexpr float kNearThresh = kNearDist * 1.002f + 1e-6f;  // conservative FP32 margin
constexpr int kNearZGroups = 32;  // warps sharing one face's z-slices (grid.y of the launch)

__device__ __forceinline__ float dot3f(float ax, float ay, float az, float bx, float by, float bz) {
    return ax * bx + ay * by + az * bz;
}

// Squared distance from p to the segment [a, a + e].
__device__ __forceinline__ float seg_d2(float px, float py, float pz, float ax, float ay, float az, float ex, float ey,
                                        float ez) {
    const float wx = px - ax, wy = py - ay, wz = pz - az;
    const float L = dot3f(ex, ey, ez, ex, ey, ez);
    float t = L > 0.f ? dot3f(wx, wy, wz, ex, ey, ez) / L : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float dx = wx - t * ex, dy = wy - t * ey, dz = wz - t * ez;
    return dot3f(dx, dy, dz, dx, dy, dz);
}

// Squared distance from p to triangle (v0, v1, v2): barycentric coordinates of the projection
// from the Gram matrix of the edges; inside -> plane distance, otherwise the nearest edge.
__device__ float tri_d2(float px, float py, float pz, const FaceRec &r) {
    const float e1x = r.r1.x - r.r0.x, e1y = r.r1.y - r.r0.y, e1z = r.r1.z - r.r0.z;
    const float e2x = r.r2.x - r.r0.x, e2y = r.r2.y - r.r0.y, e2z = r.r2.z - r.r0.z;
    const float wx = px - r.r0.x, wy = py - r.r0.y, wz = pz - r.r0.z;
    const float d00 = dot3f(e1x, e1y, e1z, e1x, e1y, e1z), d01 = dot3f(e1x, e1y, e1z, e2x, e2y, e2z);
    const float d11 = dot3f(e2x, e2y, e2z, e2x, e2y, e2z);
    const float d20 = dot3f(wx, wy, wz, e1x, e1y, e1z), d21 = dot3f(wx, wy, wz, e2x, e2y, e2z);
    const float den = d00 * d11 - d01 * d01;
    if (den > 0.f) {
        const float s = (d11 * d20 - d01 * d21) / den;
        const float t = (d00 * d21 - d01 * d20) / den;
        if (s >= 0.f && t >= 0.f && s + t <= 1.f) {
            const float dx = wx - s * e1x - t * e2x, dy = wy - s * e1y - t * e2y, dz = wz - s * e1z - t * e2z;
            return dot3f(dx, dy, dz, dx, dy, dz);
        }
    }
    const float a = seg_d2(px, py, pz, r.r0.x, r.r0.y, r.r0.z, e1x, e1y, e1z);
    const float b = seg_d2(px, py, pz, r.r1.x, r.r1.y, r.r1.z, r.r2.x - r.r1.x, r.r2.y - r.r1.y, r.r2.z - r.r1.z);
    const float c = seg_d2(px, py, pz, r.r0.x, r.r0.y, r.r0.z, e2x, e2y, e2z);
    return fminf(a, fminf(b, c));
}

__device__ __forceinline__ void index_range(float lo_box, float hi_box, float lo, float h, int n, int &i0, int &i1) {
    // voxel centres x_i = lo + (i + 0.5) h inside [lo_box, hi_box], widened by one cell for rounding
    const float a = (lo_box - lo) / h - 0.5f, b = (hi_box - lo) / h - 0.5f;
    i0 = (int)fmaxf(floorf(a) - 1.f, 0.f);
    i1 = (int)fminf(ceilf(b) + 1.f, (float)(n - 1));
}

__global__ void near_grid_kernel(const FaceRec *__restrict__ rec, int64_t nf, GridF g, uint8_t *__restrict__ flag) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float T2 = kNearThresh * kNearThresh;
    for (int64_t f = warp; f < nf; f += nwarps) {
        const FaceRec r = rec[f];
        int i0[3], i1[3];
        const float vmin[3] = {fminf(r.r0.x, fminf(r.r1.x, r.r2.x)), fminf(r.r0.y, fminf(r.r1.y, r.r2.y)),
                               fminf(r.r0.z, fminf(r.r1.z, r.r2.z))};
        const float vmax[3] = {fmaxf(r.r0.x, fmaxf(r.r1.x, r.r2.x)), fmaxf(r.r0.y, fmaxf(r.r1.y, r.r2.y)),
                               fmaxf(r.r0.z, fmaxf(r.r1.z, r.r2.z))};
        bool empty = false;
        for (int k = 0; k < 3; ++k) {
            index_range(vmin[k] - kNearThresh, vmax[k] + kNearThresh, g.lo[k], g.h[k], g.n[k], i0[k], i1[k]);
            if (i1[k] < i0[k]) empty = true;
        }
        if (empty) continue;
        const int64_t sx = i1[0] - i0[0] + 1, sy = i1[1] - i0[1] + 1;
        const int64_t total = sx * sy;
        // z-slices of the box are shared out over grid.y, so a face much larger than a voxel
        // is covered by many warps
        for (int iz = i0[2] + (int)blockIdx.y; iz <= i1[2]; iz += (int)gridDim.y) {
            const float pz = __fmaf_rn((float)iz + 0.5f, g.h[2], g.lo[2]);
            for (int64_t t = lane; t < total; t += 32) {
                const int ix = i0[0] + (int)(t % sx);
                const int iy = i0[1] + (int)(t / sx);
                const float px = __fmaf_rn((float)ix + 0.5f, g.h[0], g.lo[0]);
                const float py = __fmaf_rn((float)iy + 0.5f, g.h[1], g.lo[1]);
                const int64_t qi = ((int64_t)iz * g.n[1] + iy) * g.n[0] + ix;
                if (tri_d2(px, py, pz, r) <= T2 && DV_INB(qi, (int64_t)g.n[0] * g.n[1] * g.n[2], kSiteNear))
                    flag[qi] = 1;
            }
        }
    }
}

// List path: the queries are binned into a kBinG^3 grid of cells over the mesh's bounding box
// grown by the threshold (queries outside it cannot be near), counting-sorted by cell, and each
// face visits the cells its grown box overlaps, testing the queries there. Work is
// O(sum over faces of queries in the grown box) instead of O(Q x F).
constexpr int kBinG = 128;
constexpr int kBoxThreads = 1024;

// Grown bounding box of all faces: box[0..2] = lo, box[3..5] = hi (one CTA).
__global__ void __launch_bounds__(kBoxThreads) mesh_box_kernel(const FaceRec *__restrict__ rec, int64_t nf,
                                                               float *__restrict__ box) {
    __shared__ float red[6][kBoxThreads / 32];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t f = threadIdx.x; f < nf; f += kBoxThreads) {
        const FaceRec r = rec[f];
        const float x[3][3] = {{r.r0.x, r.r0.y, r.r0.z}, {r.r1.x, r.r1.y, r.r1.z}, {r.r2.x, r.r2.y, r.r2.z}};
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], x[v][k]);
                hi[k] = fmaxf(hi[k], x[v][k]);
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(kFull, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(kFull, hi[k], o));
        }
        if (lane == 0) {
            red[k][warp] = lo[k];
            red[3 + k][warp] = hi[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float v = red[k][0];
        for (int w = 1; w < kBoxThreads / 32; ++w) v = k < 3 ? fminf(v, red[k][w]) : fmaxf(v, red[k][w]);
        // grown by the threshold plus a relative margin for the FP32 cell arithmetic
        const float m = kNearThresh + 1e-6f * fabsf(v);
        box[k] = k < 3 ? v - m : v + m;
    }
}

__device__ __forceinline__ bool bin_coords(const float *box, float px, float py, float pz, int c[3]) {
    const float p[3] = {px, py, pz};
    for (int k = 0; k < 3; ++k) {
        if (!(p[k] >= box[k] && p[k] <= box[3 + k])) return false;
        const float t = (p[k] - box[k]) / (box[3 + k] - box[k]) * (float)kBinG;
        c[k] = min(max((int)t, 0), kBinG - 1);
    }
    return true;
}

__global__ void bin_count_kernel(const float *__restrict__ q, int64_t nq, const float *__restrict__ box,
                                 int *__restrict__ counts, int *__restrict__ qcell) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        int cell = -1;
        if (bin_coords(box, q[3 * i], q[3 * i + 1], q[3 * i + 2], c)) {
            cell = (c[2] * kBinG + c[1]) * kBinG + c[0];
            atomicAdd(&counts[cell], 1);
        }
        qcell[i] = cell;
    }
}

// Exclusive scan of the kBinG^3 counts into offsets (one CTA: each thread scans a contiguous
// chunk, the chunk totals are scanned across the CTA).
__global__ void __launch_bounds__(kBoxThreads) bin_scan_kernel(const int *__restrict__ counts,
                                                               int *__restrict__ offsets) {
    constexpr int kCells = kBinG * kBinG * kBinG;
    constexpr int kChunk = kCells / kBoxThreads;
    __shared__ int part[kBoxThreads];
    const int base = threadIdx.x * kChunk;
    int s = 0;
    for (int i = 0; i < kChunk; ++i) s += counts[base + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kBoxThreads; o <<= 1) {  // inclusive Hillis-Steele scan of the chunk totals
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int i = 0; i < kChunk; ++i) {
        offsets[base + i] = run;
        run += counts[base + i];
    }
    if (threadIdx.x == kBoxThreads - 1) offsets[kCells] = run;
}

// Queries into cell order; counts[] is consumed (decremented to 0) for the slot within the cell.
__global__ void bin_scatter_kernel(int64_t nq, const int *__restrict__ qcell, const int *__restrict__ offsets,
                                   int *__restrict__ counts, int *__restrict__ sorted) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int cell = qcell[i];
        if (cell < 0) continue;
        const int slot = atomicSub(&counts[cell], 1) - 1;
        sorted[offsets[cell] + slot] = (int)i;
    }
}

// One warp per (face, z-group of bin layers): test the queries in the bins that the face's
// grown box overlaps.
__global__ void near_binned_kernel(const FaceRec *__restrict__ rec, int64_t nf, const float *__restrict__ q, int64_t nq,
                                   const float *__restrict__ box, const int *__restrict__ offsets,
                                   const int *__restrict__ sorted, uint8_t *__restrict__ flag) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float T2 = kNearThresh * kNearThresh;
    float b[6];
    for (int k = 0; k < 6; ++k) b[k] = box[k];
    for (int64_t f = warp; f < nf; f += nwarps) {
        const FaceRec r = rec[f];
        const float vmin[3] = {fminf(r.r0.x, fminf(r.r1.x, r.r2.x)), fminf(r.r0.y, fminf(r.r1.y, r.r2.y)),
                               fminf(r.r0.z, fminf(r.r1.z, r.r2.z))};
        const float vmax[3] = {fmaxf(r.r0.x, fmaxf(r.r1.x, r.r2.x)), fmaxf(r.r0.y, fmaxf(r.r1.y, r.r2.y)),
                               fmaxf(r.r0.z, fmaxf(r.r1.z, r.r2.z))};
        int c0[3], c1[3];
        for (int k = 0; k < 3; ++k) {
            const float sc = (float)kBinG / (b[3 + k] - b[k]);
            // one bin of slack on each side covers the rounding of the bin coordinates
            c0[k] = max((int)floorf((vmin[k] - kNearThresh - b[k]) * sc) - 1, 0);
            c1[k] = min((int)floorf((vmax[k] + kNearThresh - b[k]) * sc) + 1, kBinG - 1);
        }
        const int sx = c1[0] - c0[0] + 1, sy = c1[1] - c0[1] + 1;
        for (int cz = c0[2] + (int)blockIdx.y; cz <= c1[2]; cz += (int)gridDim.y) {
            for (int t = lane; t < sx * sy; t += 32) {
                const int cell = (cz * kBinG + c0[1] + t / sx) * kBinG + c0[0] + t % sx;
                for (int j = offsets[cell]; j < offsets[cell + 1]; ++j) {
                    const int i = sorted[j];
                    if (!DV_INB(i, nq, kSiteNear)) continue;
                    if (tri_d2(q[3 * (int64_t)i], q[3 * (int64_t)i + 1], q[3 * (int64_t)i + 2], r) <= T2) flag[i] = 1;
                }
            }
        }
    }
}

int64_t near_list_scratch_ints(int64_t nq) { return 2LL * kBinG * kBinG * kBinG + 8 + 2 * nq; }

cudaError_t launch_near_surface(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                uint8_t *near_flag, int *scratch, cudaStream_t s) {
    const int64_t nfb = (nf * 32 + 255) / 256 < 16384 ? (nf * 32 + 255) / 256 : 16384;
    if (queries) {
        // scratch (near_list_scratch_ints(nq) ints): counts [G^3], offsets [G^3 + 1], box (6 floats),
        // cell per query [nq], queries in cell order [nq]
        constexpr int64_t kCells = (int64_t)kBinG * kBinG * kBinG;
        int *counts = scratch, *offsets = scratch + kCells;
        float *box = reinterpret_cast<float *>(scratch + 2 * kCells + 1);
        int *qcell = scratch + 2 * kCells + 8, *sorted = qcell + nq;
        const unsigned qb = (unsigned)((nq + 255) / 256 < 65535 ? (nq + 255) / 256 : 65535);
        prof_begin("near_surface_list", s);
        cudaError_t e = cudaMemsetAsync(counts, 0, kCells * sizeof(int), s);
        if (e != cudaSuccess) return e;
        mesh_box_kernel<<<1, kBoxThreads, 0, s>>>(rec, nf, box);
        bin_count_kernel<<<qb, 256, 0, s>>>(queries, nq, box, counts, qcell);
        bin_scan_kernel<<<1, kBoxThreads, 0, s>>>(counts, offsets);
        bin_scatter_kernel<<<qb, 256, 0, s>>>(nq, qcell, offsets, counts, sorted);
        near_binned_kernel<<<dim3((unsigned)nfb, 4), 256, 0, s>>>(rec, nf, queries, nq, box, offsets, sorted, near_flag);
        for (int k = 0; k < 5; ++k) count_launch();
        prof_end("near_surface_list", s);
    } else {
        prof_begin("near_surface_grid", s);
        // one z-group per 32 z-layers of the grid (faces spanning many layers on fine grids get
        // more warps), at most kNearZGroups
        int zg = g->n[2] / 32;
        zg = zg < 1 ? 1 : (zg > kNearZGroups ? kNearZGroups : zg);
        near_grid_kernel<<<dim3((unsigned)nfb, (unsigned)zg), 256, 0, s>>>(rec, nf, *g, near_flag);
        count_launch();
        prof_end("near_surface_grid", s);
    }
    return cudaGetLastError();
}

}  // namespace dv
