// Mesh topology on the host, once per mesh at creation: the vertex-sharing strip order of the
// faces (below), the edge-sharing face pairs of the adjoint (build_pairs) and the boundary
// edges used by the boundary form of the adjoint (build_boundary).
//
// Vertex-sharing triangle strips.
//
// The forward pass evaluates ATAN2(N, D) of Eq. (7) for every (query, face) pair; |a|, |b|, |c|
// (one square root each) and the dots a.b, b.c, c.a depend on a vertex or an edge only. When the
// faces are visited as sequential strips (u0, u1, u2, u3, ...) whose k-th face is the vertex set
// {u_k, u_k+1, u_k+2}, every face after the first of its strip brings one new vertex and two new
// edges: per (query, face) one square root and two dots instead of three of each.
//
// The face order changes nothing in the sum of Eq. (5) beyond FP32 rounding; D is symmetric in
// (a, b, c) and N is taken from the face's own normal n_f (orientation of the input face), so
// the strip's vertex order does not have to follow the face's orientation.
//
// Strips are grown greedily: start at an unused face with the fewest unused neighbours (the
// classic heuristic that keeps isolated faces from being left as singletons; a bucket queue,
// most recently touched first), try its three
// rotations, extend each forward across the edge formed by the last two vertices and then
// backward from the first edge, keep the longest. Two faces are neighbours across an edge only
// if exactly those two faces contain it (boundary and non-manifold edges end a strip); faces
// with a repeated vertex index stay singletons.
//
// Event encoding: strip (u0, ..., u_{L+1}) with faces (f0, ..., f_{L-1}) gives the events
// (u0, -1), (u1, -1), (u2, f0), ..., (u_{L+1}, f_{L-1}): every event brings a vertex, and an event
// with face index >= 0 completes the face formed with the two vertices before it.
#include <algorithm>
#include <cstdint>
#include <new>
#include <utility>
#include <vector>

#include "dv_internal.cuh"

namespace dv {

namespace {

bool degenerate(const int32_t *t) { return t[0] == t[1] || t[1] == t[2] || t[2] == t[0]; }

}  // namespace

void build_strips(const int32_t *faces, int64_t nf, int64_t nv, std::vector<int32_t> &ev_vert,
                  std::vector<int32_t> &ev_face) {
    ev_vert.clear();
    ev_face.clear();
    ev_vert.reserve((size_t)nf * 3 / 2 + 16);
    ev_face.reserve((size_t)nf * 3 / 2 + 16);
    // vertex -> incident faces (CSR), then the neighbour across each local edge (-1: none)
    std::vector<int32_t> vptr((size_t)nv + 1, 0), vfaces((size_t)nf * 3);
    for (int64_t i = 0; i < 3 * nf; ++i) vptr[(size_t)faces[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    {
        std::vector<int32_t> fill(vptr.begin(), vptr.end() - 1);
        for (int64_t i = 0; i < 3 * nf; ++i) vfaces[(size_t)fill[faces[i]]++] = (int32_t)(i / 3);
    }
    std::vector<int32_t> nb((size_t)nf * 3, -1);
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t *t = faces + 3 * f;
        if (degenerate(t)) continue;
        for (int k = 0; k < 3; ++k) {
            const int32_t u = t[k], v = t[(k + 1) % 3];
            int32_t g = -1, n_other = 0;
            for (int32_t c = vptr[u]; c < vptr[u + 1]; ++c) {
                const int32_t h = vfaces[c];
                if (h == f) continue;
                const int32_t *th = faces + 3 * (int64_t)h;
                if (th[0] == v || th[1] == v || th[2] == v) {  // h also has the edge {u, v}
                    if (h != g) ++n_other;  // (a face listed twice under u counts once)
                    g = h;
                }
            }
            if (n_other == 1 && !degenerate(faces + 3 * (int64_t)g)) nb[(size_t)f * 3 + k] = g;
        }
    }
    std::vector<uint8_t> used((size_t)nf, 0);
    std::vector<int32_t> deg((size_t)nf, 0), stamp((size_t)nf, 0);
    // bucket queue on the number of unused neighbours (0..3), stale entries skipped on pop
    std::vector<int32_t> bucket[4];
    for (int64_t f = nf - 1; f >= 0; --f) {
        for (int k = 0; k < 3; ++k) deg[f] += nb[(size_t)f * 3 + k] >= 0;
        bucket[deg[f]].push_back((int32_t)f);
    }
    int32_t cur_stamp = 0;

    // Grow (seq, fs) across the edge (seq[-2], seq[-1]) while the face there is free.
    auto extend = [&](std::vector<int32_t> &seq, std::vector<int32_t> &fs) {
        for (;;) {
            const int32_t u = seq[seq.size() - 2], v = seq[seq.size() - 1], cur = fs.back();
            const int32_t *t = faces + 3 * (int64_t)cur;
            int32_t g = -1;
            for (int k = 0; k < 3; ++k) {
                const int32_t p = t[k], q = t[(k + 1) % 3];
                if ((p == u && q == v) || (p == v && q == u)) g = nb[(size_t)cur * 3 + k];
            }
            if (g < 0 || used[g] || stamp[g] == cur_stamp) return;
            const int32_t *tg = faces + 3 * (int64_t)g;
            int32_t w = -1;
            for (int k = 0; k < 3; ++k)
                if (tg[k] != u && tg[k] != v) w = tg[k];
            if (w < 0) return;
            seq.push_back(w);
            fs.push_back(g);
            stamp[g] = cur_stamp;
        }
    };

    std::vector<int32_t> seq, fs, best_seq, best_fs;
    for (;;) {
        int32_t f = -1;
        for (int d = 0; d < 4 && f < 0; ++d) {
            while (!bucket[d].empty()) {
                const int32_t h = bucket[d].back();
                bucket[d].pop_back();
                if (!used[h] && deg[h] == d) {
                    f = h;
                    break;
                }
            }
        }
        if (f < 0) break;
        best_seq.clear();
        best_fs.clear();
        const int32_t *t = faces + 3 * (int64_t)f;
        const int rots = degenerate(t) ? 1 : 3;
        for (int r = 0; r < rots; ++r) {
            ++cur_stamp;
            seq.assign({t[r], t[(r + 1) % 3], t[(r + 2) % 3]});
            fs.assign({f});
            stamp[f] = cur_stamp;
            if (rots == 3) {
                extend(seq, fs);
                std::reverse(seq.begin(), seq.end());
                std::reverse(fs.begin(), fs.end());
                extend(seq, fs);
            }
            if (fs.size() > best_fs.size()) {
                best_seq.swap(seq);
                best_fs.swap(fs);
            }
        }
        ev_vert.push_back(best_seq[0]);
        ev_face.push_back(-1);
        ev_vert.push_back(best_seq[1]);
        ev_face.push_back(-1);
        for (size_t k = 0; k < best_fs.size(); ++k) {
            ev_vert.push_back(best_seq[k + 2]);
            ev_face.push_back(best_fs[k]);
        }
        for (const int32_t g : best_fs) used[g] = 1;
        for (const int32_t g : best_fs)
            for (int k = 0; k < 3; ++k) {
                const int32_t h = nb[(size_t)g * 3 + k];
                if (h >= 0 && !used[h]) bucket[--deg[h]].push_back(h);
            }
    }
}

// Pairs of faces that share an edge, for the adjoint (winding_bwd.cu): two consecutive
// faces of a strip share the edge formed by the two events between them, so per (query, pair)
// four vertex distances and five edge dots serve both faces instead of six and six. Faces of a
// strip are paired front to back; what is left (odd strip ends, singletons) is listed in
// `singles`. Pair record (8 ints): p0, p1, p2, p3, fA, fB, code, 0, where face A is (p0, p1, p2)
// in its own orientation (a rotation of its input corners) and face B is the vertex set
// {p1, p2, p3} taken as (p2, p1, p3); `code` holds, for the canonical corners c = 0, 1, 2 of A
// and then of B, the input corner each one is (2 bits each, A at bit 2c, B at bit 6 + 2c), and
// bit 12 when B's input orientation is the reverse of (p2, p1, p3).
void build_pairs(const int32_t *faces, int64_t nf, const std::vector<int32_t> &ev_vert,
                 const std::vector<int32_t> &ev_face, std::vector<int32_t> &pairs, std::vector<int32_t> &singles) {
    pairs.clear();
    singles.clear();
    pairs.reserve((size_t)nf * 4);
    singles.reserve((size_t)nf / 4 + 16);
    const int64_t ne = (int64_t)ev_vert.size();
    auto corner_of = [&](int32_t f, int32_t v) {
        for (int c = 0; c < 3; ++c)
            if (faces[3 * (int64_t)f + c] == v) return c;
        return -1;
    };
    for (int64_t k = 0; k < ne; ++k) {
        const int32_t fa = ev_face[(size_t)k];
        if (fa < 0) continue;
        const int32_t fb = k + 1 < ne ? ev_face[(size_t)k + 1] : -1;
        bool paired = false;
        if (fb >= 0 && k >= 2) {
            const int32_t u = ev_vert[(size_t)k - 2], s1 = ev_vert[(size_t)k - 1], s2 = ev_vert[(size_t)k],
                          w = ev_vert[(size_t)k + 1];
            const bool distinct = u != s1 && u != s2 && u != w && s1 != s2 && s1 != w && s2 != w;
            const int ra = distinct ? corner_of(fa, u) : -1;
            if (ra >= 0 && !degenerate(faces + 3 * (int64_t)fa) && !degenerate(faces + 3 * (int64_t)fb)) {
                const int32_t p1 = faces[3 * (int64_t)fa + (ra + 1) % 3], p2 = faces[3 * (int64_t)fa + (ra + 2) % 3];
                const int b0 = corner_of(fb, p2), b1 = corner_of(fb, p1), b2 = corner_of(fb, w);
                if (((p1 == s1 && p2 == s2) || (p1 == s2 && p2 == s1)) && b0 >= 0 && b1 >= 0 && b2 >= 0) {
                    const bool rev = b1 != (b0 + 1) % 3;
                    const int32_t code = ra | ((ra + 1) % 3) << 2 | ((ra + 2) % 3) << 4 | b0 << 6 | b1 << 8 |
                                         b2 << 10 | (rev ? 1 << 12 : 0);
                    const int32_t rec[8] = {u, p1, p2, w, fa, fb, code, 0};
                    pairs.insert(pairs.end(), rec, rec + 8);
                    paired = true;
                }
            }
        }
        if (paired)
            ++k;  // fb is taken
        else
            singles.push_back(fa);
    }
}

void build_boundary(const int32_t *faces, int64_t nf, int64_t nv, std::vector<int32_t> &edges,
                    std::vector<int32_t> &vptr, std::vector<int32_t> &vend) {
    // net multiplicity of every undirected edge {u < v}: +1 per face traversing u -> v, -1 per
    // v -> u. The directed edges are bucketed by their lower endpoint (CSR), each short bucket is
    // sorted by the upper endpoint and equal entries are merged, so the edges come out ordered
    // by (u, v).
    std::vector<int32_t> lptr((size_t)nv + 1, 0);
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) {
            const int32_t u = faces[3 * f + k], v = faces[3 * f + (k + 1) % 3];
            if (u != v) lptr[(size_t)(u < v ? u : v) + 1]++;  // a zero-length edge contributes nothing
        }
    for (int64_t v = 0; v < nv; ++v) lptr[v + 1] += lptr[v];
    std::vector<std::pair<int32_t, int32_t>> he((size_t)lptr[nv]);  // (upper endpoint, +-1)
    {
        std::vector<int32_t> fill(lptr.begin(), lptr.end() - 1);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) {
                const int32_t u = faces[3 * f + k], v = faces[3 * f + (k + 1) % 3];
                if (u == v) continue;
                he[(size_t)fill[u < v ? u : v]++] = {u < v ? v : u, u < v ? 1 : -1};
            }
    }
    edges.clear();
    for (int64_t lo = 0; lo < nv; ++lo) {
        auto b = he.begin() + lptr[lo], e = he.begin() + lptr[lo + 1];
        std::sort(b, e, [](const std::pair<int32_t, int32_t> &x, const std::pair<int32_t, int32_t> &y) {
            return x.first < y.first;
        });
        for (auto i = b; i != e;) {
            auto j = i;
            int32_t m = 0;
            while (j != e && j->first == i->first) m += (j++)->second;
            if (m != 0) {
                edges.push_back((int32_t)lo);
                edges.push_back(i->first);
                edges.push_back(m);
            }
            i = j;
        }
    }
    const int64_t nb = (int64_t)edges.size() / 3;
    vptr.assign((size_t)nv + 1, 0);
    for (int64_t e = 0; e < nb; ++e) {
        vptr[(size_t)edges[3 * e] + 1]++;
        vptr[(size_t)edges[3 * e + 1] + 1]++;
    }
    for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    vend.assign((size_t)nb * 2, 0);
    std::vector<int32_t> fill(vptr.begin(), vptr.end() - 1);
    for (int64_t e = 0; e < nb; ++e) {
        vend[(size_t)fill[edges[3 * e]]++] = (int32_t)(2 * e);
        vend[(size_t)fill[edges[3 * e + 1]]++] = (int32_t)(2 * e + 1);
    }
}

}  // namespace dv

extern "C" dv_status dv_build_strips(const int32_t *faces, int64_t nf, int64_t nv, int32_t *ev_vert,
                                     int32_t *ev_face, int64_t capacity, int64_t *n_events) {
    if (!faces || !n_events || nf < 1 || nv < 3 || capacity < 0)
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_build_strips: bad arguments");
    for (int64_t i = 0; i < 3 * nf; ++i)
        if (faces[i] < 0 || faces[i] >= nv)
            return dv::report_error(DV_ERR_INVALID_MESH, "dv_build_strips: face index outside [0, nv)");
    std::vector<int32_t> v, f;
    try {
        dv::build_strips(faces, nf, nv, v, f);
    } catch (const std::bad_alloc &) {
        return dv::report_error(DV_ERR_OOM, "dv_build_strips: host memory");
    }
    *n_events = (int64_t)v.size();
    if (!ev_vert || !ev_face) return DV_OK;  // size query
    if (capacity < (int64_t)v.size())
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_build_strips: capacity below the number of events");
    std::copy(v.begin(), v.end(), ev_vert);
    std::copy(f.begin(), f.end(), ev_face);
    return DV_OK;
}

extern "C" dv_status dv_build_face_pairs(const int32_t *faces, int64_t nf, int64_t nv, int32_t *pairs,
                                         int32_t *singles, int64_t capacity_pairs, int64_t capacity_singles,
                                         int64_t *n_pairs, int64_t *n_singles) {
    if (!faces || !n_pairs || !n_singles || nf < 1 || nv < 3 || capacity_pairs < 0 || capacity_singles < 0)
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_build_face_pairs: bad arguments");
    for (int64_t i = 0; i < 3 * nf; ++i)
        if (faces[i] < 0 || faces[i] >= nv)
            return dv::report_error(DV_ERR_INVALID_MESH, "dv_build_face_pairs: face index outside [0, nv)");
    std::vector<int32_t> v, f, p, sg;
    try {
        dv::build_strips(faces, nf, nv, v, f);
        dv::build_pairs(faces, nf, v, f, p, sg);
    } catch (const std::bad_alloc &) {
        return dv::report_error(DV_ERR_OOM, "dv_build_face_pairs: host memory");
    }
    *n_pairs = (int64_t)p.size() / 8;
    *n_singles = (int64_t)sg.size();
    if (!pairs || !singles) return DV_OK;  // size query
    if (capacity_pairs < *n_pairs || capacity_singles < *n_singles)
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_build_face_pairs: capacity below the count");
    std::copy(p.begin(), p.end(), pairs);
    std::copy(sg.begin(), sg.end(), singles);
    return DV_OK;
}
