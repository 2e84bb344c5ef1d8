// Vertex-sharing triangle strips of a mesh (host code, run once per mesh at creation).
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
// Strips are grown greedily: start at the unused face with the fewest unused neighbours (the
// classic heuristic that keeps isolated faces from being left as singletons), try its three
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
#include <queue>
#include <utility>
#include <vector>

#include "dv_internal.cuh"

namespace dv {

namespace {

struct Edge {
    uint64_t key;
    int32_t face;
    int32_t local;  // edge k joins corners k and (k+1) % 3
};

bool degenerate(const int32_t *t) { return t[0] == t[1] || t[1] == t[2] || t[2] == t[0]; }

}  // namespace

void build_strips(const int32_t *faces, int64_t nf, int64_t nv, std::vector<int32_t> &ev_vert,
                  std::vector<int32_t> &ev_face) {
    ev_vert.clear();
    ev_face.clear();
    ev_vert.reserve((size_t)nf * 3 / 2 + 16);
    ev_face.reserve((size_t)nf * 3 / 2 + 16);
    // neighbour across each local edge (-1: none)
    std::vector<int32_t> nb((size_t)nf * 3, -1);
    {
        std::vector<Edge> e;
        e.reserve((size_t)nf * 3);
        for (int64_t f = 0; f < nf; ++f) {
            const int32_t *t = faces + 3 * f;
            if (degenerate(t)) continue;
            for (int k = 0; k < 3; ++k) {
                const uint64_t u = (uint32_t)t[k], v = (uint32_t)t[(k + 1) % 3];
                const uint64_t key = u < v ? (u * (uint64_t)nv + v) : (v * (uint64_t)nv + u);
                e.push_back({key, (int32_t)f, k});
            }
        }
        std::sort(e.begin(), e.end(), [](const Edge &x, const Edge &y) {
            return x.key != y.key ? x.key < y.key : (x.face != y.face ? x.face < y.face : x.local < y.local);
        });
        for (size_t i = 0; i < e.size();) {
            size_t j = i;
            while (j < e.size() && e[j].key == e[i].key) ++j;
            if (j - i == 2 && e[i].face != e[i + 1].face) {
                nb[(size_t)e[i].face * 3 + e[i].local] = e[i + 1].face;
                nb[(size_t)e[i + 1].face * 3 + e[i + 1].local] = e[i].face;
            }
            i = j;
        }
    }
    std::vector<uint8_t> used((size_t)nf, 0);
    std::vector<int32_t> deg((size_t)nf, 0), stamp((size_t)nf, 0);
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) deg[f] += nb[(size_t)f * 3 + k] >= 0;
    using Item = std::pair<int32_t, int32_t>;  // (unused neighbours, face)
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int64_t f = 0; f < nf; ++f) heap.push({deg[f], (int32_t)f});
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
    while (!heap.empty()) {
        const Item it = heap.top();
        heap.pop();
        const int32_t f = it.second;
        if (used[f] || it.first != deg[f]) continue;
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
                best_seq = seq;
                best_fs = fs;
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
                if (h >= 0 && !used[h]) heap.push({--deg[h], h});
            }
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
    dv::build_strips(faces, nf, nv, v, f);
    *n_events = (int64_t)v.size();
    if (!ev_vert || !ev_face) return DV_OK;  // size query
    if (capacity < (int64_t)v.size())
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_build_strips: capacity below the number of events");
    std::copy(v.begin(), v.end(), ev_vert);
    std::copy(f.begin(), f.end(), ev_face);
    return DV_OK;
}
