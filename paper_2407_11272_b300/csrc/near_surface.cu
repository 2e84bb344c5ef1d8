// Near-surface selection for the FP64 re-evaluation: flag every query within kNearDist of a
// triangle (Euclidean distance, conservative: a small FP32 margin only adds queries).
//
// Grid path: a warp per (face, z-slice group) visits the voxel centres inside the face's
// bounding box grown by the threshold, computes the point-triangle distance in FP32 and sets
// near_flag[q] = 1.
// Work is O(sum over faces of voxels in the grown box), far below the F x Q pair count.
// List path: one thread per query scans all faces with a bounding-box reject first.
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
                if (tri_d2(px, py, pz, r) <= T2) flag[((int64_t)iz * g.n[1] + iy) * g.n[0] + ix] = 1;
            }
        }
    }
}

__global__ void near_list_kernel(const FaceRec *__restrict__ rec, int64_t nf, const float *__restrict__ q,
                                 int64_t nq, uint8_t *__restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const float px = q[3 * i], py = q[3 * i + 1], pz = q[3 * i + 2];
    const float T2 = kNearThresh * kNearThresh;
    uint8_t hit = 0;
    for (int64_t f = 0; f < nf && !hit; ++f) {
        const FaceRec r = rec[f];
        if (px < fminf(r.r0.x, fminf(r.r1.x, r.r2.x)) - kNearThresh) continue;
        if (px > fmaxf(r.r0.x, fmaxf(r.r1.x, r.r2.x)) + kNearThresh) continue;
        if (py < fminf(r.r0.y, fminf(r.r1.y, r.r2.y)) - kNearThresh) continue;
        if (py > fmaxf(r.r0.y, fmaxf(r.r1.y, r.r2.y)) + kNearThresh) continue;
        if (pz < fminf(r.r0.z, fminf(r.r1.z, r.r2.z)) - kNearThresh) continue;
        if (pz > fmaxf(r.r0.z, fmaxf(r.r1.z, r.r2.z)) + kNearThresh) continue;
        if (tri_d2(px, py, pz, r) <= T2) hit = 1;
    }
    flag[i] = hit;
}

cudaError_t launch_near_surface(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                uint8_t *near_flag, cudaStream_t s) {
    if (queries) {
        prof_begin("near_surface_list", s);
        near_list_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(rec, nf, queries, nq, near_flag);
    } else {
        prof_begin("near_surface_grid", s);
        int64_t blocks = (nf * 32 + 255) / 256;
        if (blocks > 16384) blocks = 16384;
        // one z-group per 32 z-layers of the grid (faces spanning many layers on fine grids get
        // more warps), at most kNearZGroups
        int zg = g->n[2] / 32;
        zg = zg < 1 ? 1 : (zg > kNearZGroups ? kNearZGroups : zg);
        const unsigned zgroups = (unsigned)zg;
        near_grid_kernel<<<dim3((unsigned)blocks, zgroups), 256, 0, s>>>(rec, nf, *g, near_flag);
    }
    count_launch();
    prof_end(queries ? "near_surface_list" : "near_surface_grid", s);
    return cudaGetLastError();
}

}  // namespace dv
