// Mesh validation, per-face record packing (Algorithm 1: "f_i = (v0, v1, v2)") and the
// deterministic vertex gather of the adjoint.
#include <math.h>

#include "dv_internal.cuh"

namespace dv {

__global__ void validate_kernel(const float *__restrict__ verts, int64_t nv, const int32_t *__restrict__ faces,
                                int64_t nf, int *bad) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nf; i += stride) {
        int32_t k = faces[i];
        if (k < 0 || (int64_t)k >= nv) atomicCAS(bad, 0, 1);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nv; i += stride) {
        if (!isfinite(verts[i])) atomicCAS(bad, 0, 2);
    }
}

// Per face: gather the three vertices, compute n = (v1 - v0) x (v2 - v0) in FP64 (products of
// FP32 values are exact in FP64), and store the FP32 record (normal scaled by 8) and the FP64
// record used by the re-evaluation pass.
__device__ __forceinline__ void pack_one(const float *__restrict__ verts, int64_t nv, const int32_t *__restrict__ faces,
                                         int64_t f, FaceRec *__restrict__ rec, FaceRec64 *__restrict__ rec64) {
    double v[3][3];
    for (int k = 0; k < 3; ++k) {
        int64_t id = faces[3 * f + k];
        if (!DV_INB(id, nv, kSitePack)) id = 0;
        for (int c = 0; c < 3; ++c) v[k][c] = (double)verts[3 * id + c];
    }
    double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    FaceRec r;
    r.r0 = make_float4((float)v[0][0], (float)v[0][1], (float)v[0][2], (float)(kNormalScale * n[0]));
    r.r1 = make_float4((float)v[1][0], (float)v[1][1], (float)v[1][2], (float)(kNormalScale * n[1]));
    r.r2 = make_float4((float)v[2][0], (float)v[2][1], (float)v[2][2], (float)(kNormalScale * n[2]));
    rec[f] = r;
    FaceRec64 r64;
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) r64.v[3 * k + c] = v[k][c];
    for (int c = 0; c < 3; ++c) r64.v[9 + c] = n[c];
    rec64[f] = r64;
}

__global__ void pack_kernel(const float *__restrict__ verts, int64_t nv, const int32_t *__restrict__ faces, int64_t nf,
                            FaceRec *__restrict__ rec, FaceRec64 *__restrict__ rec64) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x)
        pack_one(verts, nv, faces, f, rec, rec64);
}

// dverts[v] = sum over the faces f incident to v (corner k) and over the query splits s of
// face_grad[s][f][3k..3k+2], summed in FP64 in a fixed order (deterministic).
__global__ void gather_dverts_kernel(const float *__restrict__ face_grad, int nsplit, int64_t nf,
                                     const int32_t *__restrict__ vtx_ptr, const int32_t *__restrict__ vtx_corner,
                                     int64_t nv, float *__restrict__ dverts) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int32_t c = vtx_ptr[v]; c < vtx_ptr[v + 1]; ++c) {
        if (!DV_INB(c, 3 * nf, kSiteGather)) break;
        int32_t corner = vtx_corner[c];
        if (!DV_INB(corner, 3 * nf, kSiteGather)) continue;
        int64_t f = corner / 3;
        int k = corner - 3 * (int)f;
        for (int s = 0; s < nsplit; ++s) {
            const float *g = face_grad + ((int64_t)s * nf + f) * 9 + 3 * k;
            s0 += (double)g[0];
            s1 += (double)g[1];
            s2 += (double)g[2];
        }
    }
    dverts[3 * v + 0] = (float)s0;
    dverts[3 * v + 1] = (float)s1;
    dverts[3 * v + 2] = (float)s2;
}

// The same sum with a warp per vertex when there are many splits (small meshes on many row
// splits): lane l takes splits l, l + 32, ... of every incident (face, corner) in CSR order, then
// a fixed butterfly over the lanes; deterministic for a given split count.
__global__ void gather_dverts_warp_kernel(const float *__restrict__ face_grad, int nsplit, int64_t nf,
                                          const int32_t *__restrict__ vtx_ptr,
                                          const int32_t *__restrict__ vtx_corner, int64_t nv,
                                          float *__restrict__ dverts) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += warps) {  // whole warps
        double s0 = 0, s1 = 0, s2 = 0;
        for (int32_t c = vtx_ptr[v]; c < vtx_ptr[v + 1]; ++c) {
            if (!DV_INB(c, 3 * nf, kSiteGather)) break;
            const int32_t corner = vtx_corner[c];
            if (!DV_INB(corner, 3 * nf, kSiteGather)) continue;
            const int64_t f = corner / 3;
            const int k = corner - 3 * (int)f;
            for (int s = lane; s < nsplit; s += 32) {
                const float *g = face_grad + ((int64_t)s * nf + f) * 9 + 3 * k;
                s0 += (double)g[0];
                s1 += (double)g[1];
                s2 += (double)g[2];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            dverts[3 * v + 0] = (float)s0;
            dverts[3 * v + 1] = (float)s1;
            dverts[3 * v + 2] = (float)s2;
        }
    }
}

static int blocks_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_validate(const float *verts, int64_t nv, const int32_t *faces, int64_t nf, int *d_bad,
                            cudaStream_t s) {
    prof_begin("validate_mesh", s);
    validate_kernel<<<blocks_for(3 * (nf > nv ? nf : nv), 256, 4096), 256, 0, s>>>(verts, nv, faces, nf, d_bad);
    count_launch();
    prof_end("validate_mesh", s);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *verts, int64_t nv, const int32_t *faces, int64_t nf, FaceRec *rec,
                        FaceRec64 *rec64, cudaStream_t s) {
    prof_begin("pack_faces", s);
    pack_kernel<<<blocks_for(nf, 256), 256, 0, s>>>(verts, nv, faces, nf, rec, rec64);
    count_launch();
    prof_end("pack_faces", s);
    return cudaGetLastError();
}

// One strip event: the vertex (FP32 as given, and widened to FP64) and, for an event that
// completes a face, that face's normal taken from the packed face records.
__device__ __forceinline__ void pack_strip_one(const float *__restrict__ verts, int64_t nv, int64_t nf,
                                               const int32_t *__restrict__ ev_vert, const int32_t *__restrict__ ev_face,
                                               int64_t e,
                                               const FaceRec *__restrict__ rec, const FaceRec64 *__restrict__ rec64,
                                               StripRec *__restrict__ srec, StripRec64 *__restrict__ srec64) {
    int64_t v = ev_vert[e];
    int32_t f = ev_face[e];
    if (!DV_INB(v, nv, kSitePack)) v = 0;
    if (f >= 0 && !DV_INB(f, nf, kSitePack)) f = -1;
    const float x = verts[3 * v], y = verts[3 * v + 1], z = verts[3 * v + 2];
    StripRec r;
    StripRec64 r64;
    r64.v[0] = x;
    r64.v[1] = y;
    r64.v[2] = z;
    r64.pad = 0.0;
    if (f >= 0) {
        const FaceRec fr = rec[f];
        r.p = make_float4(x, y, z, fr.r0.w);
        r.q = make_float4(fr.r1.w, fr.r2.w, 1.0f, 0.0f);
        for (int c = 0; c < 3; ++c) r64.n[c] = rec64[f].v[9 + c];
        r64.flag = 1.0;
    } else {
        r.p = make_float4(x, y, z, 0.0f);
        r.q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int c = 0; c < 3; ++c) r64.n[c] = 0.0;
        r64.flag = 0.0;
    }
    srec[e] = r;
    srec64[e] = r64;
}

__global__ void pack_strips_kernel(const float *__restrict__ verts, int64_t nv, int64_t nf,
                                   const int32_t *__restrict__ ev_vert,
                                   const int32_t *__restrict__ ev_face, int64_t ne, const FaceRec *__restrict__ rec,
                                   const FaceRec64 *__restrict__ rec64, StripRec *__restrict__ srec,
                                   StripRec64 *__restrict__ srec64) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
        pack_strip_one(verts, nv, nf, ev_vert, ev_face, e, rec, rec64, srec, srec64);
}

cudaError_t launch_pack_strips(const float *verts, int64_t nv, int64_t nf, const int32_t *ev_vert,
                               const int32_t *ev_face, int64_t ne, const FaceRec *rec, const FaceRec64 *rec64,
                               StripRec *srec, StripRec64 *srec64, cudaStream_t s) {
    if (ne == 0) return cudaSuccess;
    prof_begin("pack_strips", s);
    pack_strips_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(verts, nv, nf, ev_vert, ev_face, ne, rec, rec64, srec,
                                                           srec64);
    count_launch();
    prof_end("pack_strips", s);
    return cudaGetLastError();
}

// Pair records (canonical A = (p0, p1, p2), B = (p2, p1, p3)) from the packed face records:
// the vertices of A in the rotation the topology code names, p3 from B, the normals unscaled
// (8 n / 8 is exact) and B's negated when its input orientation is reversed.
__device__ __forceinline__ float4 rec_corner(const FaceRec &r, int c) { return c == 0 ? r.r0 : (c == 1 ? r.r1 : r.r2); }

__global__ void pack_pairs_kernel(const FaceRec *__restrict__ rec, const int32_t *__restrict__ ptopo, int64_t np,
                                  PairRec *__restrict__ prec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *t = ptopo + 8 * i;
        const int code = t[6];
        const FaceRec A = rec[t[4]], B = rec[t[5]];
        const float4 c0 = rec_corner(A, code & 3), c1 = rec_corner(A, (code >> 2) & 3),
                     c2 = rec_corner(A, (code >> 4) & 3), c3 = rec_corner(B, (code >> 10) & 3);
        const float inv = 1.0f / kNormalScale, sb = (code >> 12) & 1 ? -inv : inv;
        PairRec r;
        r.r0 = make_float4(c0.x, c0.y, c0.z, A.r0.w * inv);
        r.r1 = make_float4(c1.x, c1.y, c1.z, A.r1.w * inv);
        r.r2 = make_float4(c2.x, c2.y, c2.z, A.r2.w * inv);
        r.r3 = make_float4(c3.x, c3.y, c3.z, B.r0.w * sb);
        r.r4 = make_float4(B.r1.w * sb, B.r2.w * sb, 0.0f, 0.0f);
        prec[i] = r;
    }
}

cudaError_t launch_pack_pairs(const FaceRec *rec, const int32_t *ptopo, int64_t np, PairRec *prec, cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    prof_begin("pack_pairs", s);
    pack_pairs_kernel<<<blocks_for(np, 256), 256, 0, s>>>(rec, ptopo, np, prec);
    count_launch();
    prof_end("pack_pairs", s);
    return cudaGetLastError();
}

cudaError_t launch_gather_dverts(const double *, const float *face_grad, int nsplit, int64_t nf,
                                 const int32_t *vtx_ptr, const int32_t *vtx_corner, int64_t nv, float *dverts,
                                 cudaStream_t s) {
    prof_begin("gather_dverts", s);
    if (nsplit > 32)
        gather_dverts_warp_kernel<<<blocks_for(nv * 32, 256), 256, 0, s>>>(face_grad, nsplit, nf, vtx_ptr, vtx_corner,
                                                                         nv, dverts);
    else
        gather_dverts_kernel<<<blocks_for(nv, 256), 256, 0, s>>>(face_grad, nsplit, nf, vtx_ptr, vtx_corner, nv,
                                                                 dverts);
    count_launch();
    prof_end("gather_dverts", s);
    return cudaGetLastError();
}

}  // namespace dv

namespace dv {

// Algorithm 2 (Flipping Duplication), vertex part: N_v = normalized sum over the faces incident
// to v of (v1 - v0) x (v2 - v0) (area-weighted normal; the paper does not say how N_v is
// computed), summed in FP64 in the adjacency's face order. Writes v (copy) and v' = v - eps N_v.
__global__ void flipdup_verts_kernel(const float *__restrict__ verts, int64_t nv, const FaceRec64 *__restrict__ rec64,
                                     const int32_t *__restrict__ vtx_ptr, const int32_t *__restrict__ vtx_corner,
                                     double eps, float *__restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double n0 = 0, n1 = 0, n2 = 0;
    for (int32_t c = vtx_ptr[v]; c < vtx_ptr[v + 1]; ++c) {
        const FaceRec64 &r = rec64[vtx_corner[c] / 3];
        n0 += r.v[9];
        n1 += r.v[10];
        n2 += r.v[11];
    }
    const double len = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const double inv = len > 0.0 ? 1.0 / len : 0.0;
    const double p0 = verts[3 * v], p1 = verts[3 * v + 1], p2 = verts[3 * v + 2];
    out[3 * v] = (float)p0;
    out[3 * v + 1] = (float)p1;
    out[3 * v + 2] = (float)p2;
    out[3 * (nv + v)] = (float)(p0 - eps * n0 * inv);
    out[3 * (nv + v) + 1] = (float)(p1 - eps * n1 * inv);
    out[3 * (nv + v) + 2] = (float)(p2 - eps * n2 * inv);
}

// Face part: F followed by F' = {(v0', v2', v1')}: copies indexed into V', orientation reversed.
__global__ void flipdup_faces_kernel(const int32_t *__restrict__ faces, int64_t nf, int32_t nv,
                                     int32_t *__restrict__ out) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    out[3 * f] = a;
    out[3 * f + 1] = b;
    out[3 * f + 2] = c;
    out[3 * (nf + f)] = a + nv;
    out[3 * (nf + f) + 1] = c + nv;
    out[3 * (nf + f) + 2] = b + nv;
}

cudaError_t launch_flipped_duplication(const float *verts, int64_t nv, const int32_t *faces, int64_t nf,
                                       const FaceRec64 *rec64, const int32_t *vtx_ptr, const int32_t *vtx_corner,
                                       double eps, float *out_verts, int32_t *out_faces, cudaStream_t s) {
    prof_begin("flipdup_verts", s);
    flipdup_verts_kernel<<<blocks_for(nv, 256), 256, 0, s>>>(verts, nv, rec64, vtx_ptr, vtx_corner, eps, out_verts);
    count_launch();
    prof_end("flipdup_verts", s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin("flipdup_faces", s);
    flipdup_faces_kernel<<<blocks_for(nf, 256), 256, 0, s>>>(faces, nf, (int32_t)nv, out_faces);
    count_launch();
    prof_end("flipdup_faces", s);
    return cudaGetLastError();
}

}  // namespace dv
