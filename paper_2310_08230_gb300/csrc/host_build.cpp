// Host compiler: meshes + pair costs + candidate mask -> ILP (P) -> presolve -> BDD segments.
//
// Passages followed:
//  * matching elements triangle-triangle, triangle-edge, triangle-vertex with at least one
//    triangle each (Sec. 3.1, Fig. 2); about 21 |T_X||T_Y| of them (App. B);
//  * closedness rows A^d x = 0 and projection rows A^X x = 1, A^Y x = 1 (Sec. 3.1, Eq. P);
//  * a row becomes a reduced BDD without skipping arcs whose shortest path solves the row's
//    subproblem (Sec. 3.2, App. A.3); rows longer than the chunk size are split into
//    segments joined by one-hot auxiliary variables y_j = 1 iff node j of the cut layer is
//    used (App. A.3, Alg. 3, Fig. BDD);
//  * same-genus precondition (Sec. 4 "Datasets").
//
// Readings (the paper defers the product-space details to its citation): elements are
// ordered by type (tri-tri, X-tri x Y-edge, X-edge x Y-tri, X-tri x Y-vertex,
// X-vertex x Y-tri), then X element, Y element, rotation / edge pattern; a closedness row
// per product edge, +1 for an element crossing it from its lexicographically smaller
// product vertex (m, n), -1 otherwise; presolve fixes every variable some row forces
// (generalised arc consistency to a fixpoint); c_p = mean of the three pair costs,
// normalised by the largest kept c_p; segments are balanced (cut at floor(s n / S)).
//
// For a +-1 row with residual right-hand side r, the nodes of layer l are the partial sums
// sigma of the first l variables that are reachable from 0 and from which r is reachable:
// sigma in [max(-Q_pre, r - P_suf), min(P_pre, r + Q_suf)] (P / Q: counts of +1 / -1
// coefficients before / from layer l). Node s of a layer stands for sigma = lo + s.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <thread>
#include <utility>

#include "../../include/disco.h"
#include "plan.h"

namespace disco {
namespace {

// vertex sequence of a degenerate triangle over an edge (a < b): 0 -> a, 1 -> b
const int kEdgePattern[6][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

struct MeshTopo {
    int nv = 0, nt = 0;
    const int32_t* T = nullptr;
    std::vector<std::pair<int, int>> edges;     // sorted unique (a < b)
    std::vector<std::vector<std::pair<int, int>>> tri_at;  // vertex -> (triangle, corner)
    std::vector<std::vector<int>> edge_at;      // vertex -> incident edges
};

int topo(const MeshIn& m, MeshTopo* t, int* chi, std::string* err) {
    if (m.nv <= 0 || m.nt <= 0 || !m.T) { *err = "empty mesh"; return DISCO_ERR_INVALID_ARG; }
    t->nv = m.nv;
    t->nt = m.nt;
    t->T = m.T;
    std::vector<uint64_t> dir;
    dir.reserve(size_t(3) * m.nt);
    for (int f = 0; f < m.nt; ++f)
        for (int k = 0; k < 3; ++k) {
            int a = m.T[3 * f + k], b = m.T[3 * f + (k + 1) % 3];
            if (a < 0 || a >= m.nv || b < 0 || b >= m.nv) { *err = "vertex index out of range"; return DISCO_ERR_INVALID_ARG; }
            if (a == b) { *err = "degenerate triangle"; return DISCO_ERR_NONMANIFOLD; }
            dir.push_back((uint64_t(uint32_t(a)) << 32) | uint32_t(b));
        }
    std::sort(dir.begin(), dir.end());
    for (size_t i = 1; i < dir.size(); ++i)
        if (dir[i] == dir[i - 1]) { *err = "directed edge used twice (non-manifold or flipped triangle)"; return DISCO_ERR_NONMANIFOLD; }
    for (uint64_t e : dir) {
        uint64_t rev = (e << 32) | (e >> 32);
        if (!std::binary_search(dir.begin(), dir.end(), rev)) { *err = "boundary edge (open mesh)"; return DISCO_ERR_NONMANIFOLD; }
        uint32_t a = uint32_t(e >> 32), b = uint32_t(e);
        if (a < b) t->edges.emplace_back(int(a), int(b));
    }
    std::vector<char> used(m.nv, 0);
    for (int i = 0; i < 3 * m.nt; ++i) used[m.T[i]] = 1;
    for (int v = 0; v < m.nv; ++v)
        if (!used[v]) { *err = "isolated vertex"; return DISCO_ERR_NONMANIFOLD; }
    *chi = m.nv - int(t->edges.size()) + m.nt;
    t->tri_at.assign(m.nv, {});
    for (int f = 0; f < m.nt; ++f)
        for (int k = 0; k < 3; ++k) t->tri_at[m.T[3 * f + k]].emplace_back(f, k);
    t->edge_at.assign(m.nv, {});
    for (int e = 0; e < int(t->edges.size()); ++e) {
        t->edge_at[t->edges[e].first].push_back(e);
        t->edge_at[t->edges[e].second].push_back(e);
    }
    return DISCO_OK;
}

struct Elems {  // matching elements, structure of arrays
    std::vector<int32_t> m, n;  // 3 per element
    std::vector<uint8_t> type;
    std::vector<int32_t> xe, ye;
    void push(int m0, int m1, int m2, int n0, int n1, int n2, int ty, int x, int y) {
        m.push_back(m0); m.push_back(m1); m.push_back(m2);
        n.push_back(n0); n.push_back(n1); n.push_back(n2);
        type.push_back(uint8_t(ty));
        xe.push_back(x);
        ye.push_back(y);
    }
    void append(const Elems& o) {
        m.insert(m.end(), o.m.begin(), o.m.end());
        n.insert(n.end(), o.n.begin(), o.n.end());
        type.insert(type.end(), o.type.begin(), o.type.end());
        xe.insert(xe.end(), o.xe.begin(), o.xe.end());
        ye.insert(ye.end(), o.ye.begin(), o.ye.end());
    }
    size_t size() const { return type.size(); }
};

struct Allowed {
    const uint8_t* mask;  // nullptr: every pair
    int nvx, nvy;
    std::vector<std::vector<int>> row;  // m -> allowed n, ascending
    bool operator()(int a, int b) const { return !mask || mask[size_t(a) * nvy + b]; }
};

// Runs body(lo, hi, out) over [0, n) in contiguous chunks on up to `threads` threads and
// concatenates the per-chunk outputs in order (the result does not depend on threads).
template <class F>
void chunked(int n, int threads, Elems* out, F body) {
    int nch = std::max(1, std::min(threads, n / 64 + 1));
    std::vector<Elems> parts(nch);
    std::vector<std::thread> pool;
    for (int c = 0; c < nch; ++c) {
        int lo = int(int64_t(n) * c / nch), hi = int(int64_t(n) * (c + 1) / nch);
        if (nch == 1) body(lo, hi, &parts[c]);
        else pool.emplace_back([&, lo, hi, c] { body(lo, hi, &parts[c]); });
    }
    for (auto& th : pool) th.join();
    for (auto& p : parts) out->append(p);
}

void enumerate(const MeshTopo& X, const MeshTopo& Y, const Allowed& A, int threads, Elems* out) {
    const int32_t* TX = X.T;
    const int32_t* TY = Y.T;
    // type 0: X triangle t, Y triangle s, rotation r: corner v -> (t_v, s_{(v+r)%3})
    chunked(X.nt, threads, out, [&](int lo, int hi, Elems* o) {
        std::vector<int64_t> cand;
        for (int t = lo; t < hi; ++t) {
            int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
            cand.clear();
            for (int n0 : A.row[m0])
                for (auto [s, r] : Y.tri_at[n0])
                    if (A(m1, TY[3 * s + (r + 1) % 3]) && A(m2, TY[3 * s + (r + 2) % 3])) cand.push_back(int64_t(s) * 3 + r);
            std::sort(cand.begin(), cand.end());
            for (int64_t c : cand) {
                int s = int(c / 3), r = int(c % 3);
                o->push(m0, m1, m2, TY[3 * s + r], TY[3 * s + (r + 1) % 3], TY[3 * s + (r + 2) % 3], 0, t, s);
            }
        }
    });
    // type 1: X triangle t, Y edge e = (a < b), pattern p: corner v -> (t_v, pattern symbol)
    chunked(X.nt, threads, out, [&](int lo, int hi, Elems* o) {
        std::vector<int64_t> cand;
        for (int t = lo; t < hi; ++t) {
            int m[3] = {TX[3 * t], TX[3 * t + 1], TX[3 * t + 2]};
            cand.clear();
            for (int n0 : A.row[m[0]])
                for (int e : Y.edge_at[n0]) {
                    int ab[2] = {Y.edges[e].first, Y.edges[e].second};
                    for (int p = 0; p < 6; ++p)
                        if (ab[kEdgePattern[p][0]] == n0 && A(m[1], ab[kEdgePattern[p][1]]) && A(m[2], ab[kEdgePattern[p][2]]))
                            cand.push_back(int64_t(e) * 6 + p);
                }
            std::sort(cand.begin(), cand.end());
            for (int64_t c : cand) {
                int e = int(c / 6), p = int(c % 6);
                int ab[2] = {Y.edges[e].first, Y.edges[e].second};
                o->push(m[0], m[1], m[2], ab[kEdgePattern[p][0]], ab[kEdgePattern[p][1]], ab[kEdgePattern[p][2]], 1, t, e);
            }
        }
    });
    // type 2: X edge e = (a < b), Y triangle s, pattern p: corner v -> (pattern symbol, s_v)
    chunked(int(X.edges.size()), threads, out, [&](int lo, int hi, Elems* o) {
        std::vector<int64_t> cand;
        for (int e = lo; e < hi; ++e) {
            int ab[2] = {X.edges[e].first, X.edges[e].second};
            cand.clear();
            for (int p = 0; p < 6; ++p) {
                int x0 = ab[kEdgePattern[p][0]], x1 = ab[kEdgePattern[p][1]], x2 = ab[kEdgePattern[p][2]];
                for (int n0 : A.row[x0])
                    for (auto [s, r] : Y.tri_at[n0])
                        if (r == 0 && A(x1, TY[3 * s + 1]) && A(x2, TY[3 * s + 2])) cand.push_back(int64_t(s) * 6 + p);
            }
            std::sort(cand.begin(), cand.end());
            for (int64_t c : cand) {
                int s = int(c / 6), p = int(c % 6);
                o->push(ab[kEdgePattern[p][0]], ab[kEdgePattern[p][1]], ab[kEdgePattern[p][2]], TY[3 * s], TY[3 * s + 1],
                        TY[3 * s + 2], 2, e, s);
            }
        }
    });
    // type 3: X triangle t, Y vertex n
    chunked(X.nt, threads, out, [&](int lo, int hi, Elems* o) {
        for (int t = lo; t < hi; ++t) {
            int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
            for (int n : A.row[m0])
                if (A(m1, n) && A(m2, n)) o->push(m0, m1, m2, n, n, n, 3, t, n);
        }
    });
    // type 4: X vertex m, Y triangle s
    chunked(X.nv, threads, out, [&](int lo, int hi, Elems* o) {
        std::vector<int> cand;
        for (int mv = lo; mv < hi; ++mv) {
            cand.clear();
            for (int n0 : A.row[mv])
                for (auto [s, r] : Y.tri_at[n0])
                    if (r == 0 && A(mv, TY[3 * s + 1]) && A(mv, TY[3 * s + 2])) cand.push_back(s);
            std::sort(cand.begin(), cand.end());
            for (int s : cand) o->push(mv, mv, mv, TY[3 * s], TY[3 * s + 1], TY[3 * s + 2], 4, mv, s);
        }
    });
}

// Stable LSD radix sort of (key, payload) by key.
void radix_sort(std::vector<uint64_t>& key, std::vector<uint32_t>& val) {
    size_t n = key.size();
    uint64_t mx = 0;
    for (uint64_t k : key) mx = std::max(mx, k);
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> v2(n);
    for (int shift = 0; shift < 64 && (mx >> shift); shift += 16) {
        std::vector<size_t> cnt(65537, 0);
        for (size_t i = 0; i < n; ++i) ++cnt[((key[i] >> shift) & 0xFFFF) + 1];
        for (int b = 0; b < 65536; ++b) cnt[b + 1] += cnt[b];
        for (size_t i = 0; i < n; ++i) {
            size_t p = cnt[(key[i] >> shift) & 0xFFFF]++;
            k2[p] = key[i];
            v2[p] = val[i];
        }
        key.swap(k2);
        val.swap(v2);
    }
}

}  // namespace

int build_plan(const MeshIn& Xin, const MeshIn& Yin, const float* d, const uint8_t* mask, int split_chunk,
               int threads, Plan* P, std::string* err) {
    auto t0 = std::chrono::steady_clock::now();
    if (threads <= 0) threads = std::max(1u, std::thread::hardware_concurrency());
    MeshTopo X, Y;
    int chiX = 0, chiY = 0;
    int rc = topo(Xin, &X, &chiX, err);
    if (rc) { *err = "mesh X: " + *err; return rc; }
    rc = topo(Yin, &Y, &chiY, err);
    if (rc) { *err = "mesh Y: " + *err; return rc; }
    if (chiX != chiY) { *err = "Euler characteristics differ"; return DISCO_ERR_GENUS_MISMATCH; }
    const int nvx = X.nv, nvy = Y.nv;
    P->nvx = nvx;
    P->nvy = nvy;

    // ---- candidate rows
    Allowed A{mask, nvx, nvy, {}};
    A.row.assign(nvx, {});
    for (int m = 0; m < nvx; ++m)
        for (int n = 0; n < nvy; ++n)
            if (A(m, n)) A.row[m].push_back(n);

    // ---- product space
    Elems E;
    enumerate(X, Y, A, threads, &E);
    const int64_t nv = int64_t(E.size());
    if (nv == 0) { *err = "empty product space"; return DISCO_ERR_INFEASIBLE; }
    if (nv >= (int64_t(1) << 31)) { *err = "product space too large"; return DISCO_ERR_INVALID_ARG; }
    P->nvars = nv;
    P->vm = std::move(E.m);
    P->vn = std::move(E.n);

    // ---- costs: mean of the three pair costs, normalised by the largest
    P->cost.resize(nv);
    double cmax = 0.0;
    for (int64_t i = 0; i < nv; ++i) {
        double c = 0.0;
        for (int v = 0; v < 3; ++v) c += double(d[size_t(P->vm[3 * i + v]) * nvy + P->vn[3 * i + v]]);
        c /= 3.0;
        if (!(c >= 0.0) || c > 3.0e38) { *err = "pair costs must be finite and >= 0"; return DISCO_ERR_INVALID_ARG; }
        P->cost[i] = c;
        cmax = std::max(cmax, c);
    }
    if (cmax > 0)
        for (double& c : P->cost) c /= cmax;

    // ---- closedness rows: product edge (p, q), p < q in (m, n) order
    const uint64_t K = uint64_t(nvx) * uint64_t(nvy);
    std::vector<uint64_t> key(size_t(3) * nv);
    std::vector<uint32_t> pay(size_t(3) * nv);
    for (int64_t i = 0; i < nv; ++i)
        for (int v = 0; v < 3; ++v) {
            int w = (v + 1) % 3;
            uint64_t a = uint64_t(P->vm[3 * i + v]) * nvy + P->vn[3 * i + v];
            uint64_t b = uint64_t(P->vm[3 * i + w]) * nvy + P->vn[3 * i + w];
            key[3 * i + v] = std::min(a, b) * K + std::max(a, b);
            pay[3 * i + v] = uint32_t(i) * 2u + (a < b ? 0u : 1u);
        }
    radix_sort(key, pay);
    P->row_ptr.clear();
    P->row_var.resize(key.size());
    P->row_coef.resize(key.size());
    for (size_t e = 0; e < key.size(); ++e) {
        if (e == 0 || key[e] != key[e - 1]) P->row_ptr.push_back(int64_t(e));
        P->row_var[e] = int32_t(pay[e] >> 1);
        P->row_coef[e] = (pay[e] & 1u) ? -1 : 1;
    }
    P->n_closed = int64_t(P->row_ptr.size());
    P->rhs.assign(size_t(P->n_closed), 0);
    key.clear(); key.shrink_to_fit();
    pay.clear(); pay.shrink_to_fit();

    // ---- projection rows (counting sort keeps variable order inside a row)
    for (int side = 0; side < 2; ++side) {
        int ntri = side == 0 ? X.nt : Y.nt;
        std::vector<int64_t> cnt(ntri + 1, 0);
        auto tri_of = [&](int64_t i) -> int {
            int ty = E.type[i];
            if (side == 0) return (ty == 0 || ty == 1 || ty == 3) ? E.xe[i] : -1;
            return (ty == 0 || ty == 2 || ty == 4) ? E.ye[i] : -1;
        };
        for (int64_t i = 0; i < nv; ++i) {
            int t = tri_of(i);
            if (t >= 0) ++cnt[t + 1];
        }
        for (int t = 0; t < ntri; ++t)
            if (cnt[t + 1] == 0) { *err = "a triangle has no matching element"; return DISCO_ERR_INFEASIBLE; }
        for (int t = 0; t < ntri; ++t) cnt[t + 1] += cnt[t];
        int64_t base = int64_t(P->row_var.size());
        P->row_var.resize(size_t(base + cnt[ntri]));
        P->row_coef.resize(size_t(base + cnt[ntri]), 1);
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < nv; ++i) {
            int t = tri_of(i);
            if (t >= 0) P->row_var[size_t(base + pos[t]++)] = int32_t(i);
        }
        for (int t = 0; t < ntri; ++t) P->row_ptr.push_back(base + cnt[t]);
        P->rhs.resize(P->rhs.size() + size_t(ntri), 1);
        (side == 0 ? P->n_projx : P->n_projy) = ntri;
    }
    P->nrows = int64_t(P->rhs.size());
    P->row_ptr.push_back(int64_t(P->row_var.size()));

    // ---- presolve: saturated rows force all their free variables, to a fixpoint
    const int64_t nr = P->nrows;
    std::vector<int64_t> vptr(nv + 1, 0);
    for (int32_t v : P->row_var) ++vptr[v + 1];
    for (int64_t i = 0; i < nv; ++i) vptr[i + 1] += vptr[i];
    std::vector<int64_t> vrow(P->row_var.size());
    std::vector<int8_t> vcoef(P->row_var.size());
    {
        std::vector<int64_t> fill(vptr.begin(), vptr.end() - 1);
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
                int64_t p = fill[P->row_var[e]]++;
                vrow[p] = r;
                vcoef[p] = P->row_coef[e];
            }
    }
    std::vector<int32_t> res(P->rhs.begin(), P->rhs.end()), npos(nr, 0), nneg(nr, 0);
    for (int64_t r = 0; r < nr; ++r)
        for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) (P->row_coef[e] > 0 ? npos : nneg)[r]++;
    P->fixed.assign(nv, -1);
    std::vector<int64_t> queue(nr);
    std::iota(queue.begin(), queue.end(), 0);
    std::vector<char> inq(nr, 1);
    size_t head = 0;
    while (head < queue.size()) {
        int64_t r = queue[head++];
        inq[r] = 0;
        if (res[r] > npos[r] || res[r] < -nneg[r]) { *err = "presolve: a row has no solution"; return DISCO_ERR_INFEASIBLE; }
        if (npos[r] + nneg[r] == 0) continue;
        int up;  // value forced on +1 variables (-1 variables get the opposite)
        if (res[r] == npos[r]) up = 1;
        else if (res[r] == -nneg[r]) up = 0;
        else continue;
        for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
            int32_t v = P->row_var[e];
            if (P->fixed[v] >= 0) continue;
            int val = P->row_coef[e] > 0 ? up : 1 - up;
            P->fixed[v] = int8_t(val);
            for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) {
                int64_t rr = vrow[q];
                if (vcoef[q] > 0) --npos[rr]; else --nneg[rr];
                res[rr] -= vcoef[q] * val;
                if (!inq[rr]) { inq[rr] = 1; queue.push_back(rr); }
            }
        }
    }
    for (int64_t r = 0; r < nr; ++r)
        if (npos[r] + nneg[r] == 0 && res[r] != 0) { *err = "presolve: violated row"; return DISCO_ERR_INFEASIBLE; }
    P->constant = 0.0;
    std::vector<int32_t> internal(nv, -1);
    P->free_orig.clear();
    for (int64_t i = 0; i < nv; ++i) {
        if (P->fixed[i] == 1) P->constant += P->cost[i];
        if (P->fixed[i] < 0) {
            internal[i] = int32_t(P->free_orig.size());
            P->free_orig.push_back(int32_t(i));
        }
    }
    P->n_free = int64_t(P->free_orig.size());

    // ---- BDD segments
    P->slot_var.clear();
    P->slot_desc.clear();
    P->segs.clear();
    std::vector<int32_t> fv;   // free variables of a row (internal ids)
    std::vector<int8_t> fc;    // their coefficients
    std::vector<int32_t> lo, wd;
    std::vector<int32_t> slot_w, slot_wn, slot_d0, slot_d1;
    std::vector<uint8_t> slot_one;
    int64_t next_aux = 0;
    int64_t nodes = 0;
    int max_layers = 0, max_width = 0;
    auto add_slot = [&](int32_t var, int w, int wn, int d0, int d1, bool one) {
        P->slot_var.push_back(var);
        slot_w.push_back(w);
        slot_wn.push_back(wn);
        slot_d0.push_back(d0);
        slot_d1.push_back(d1);
        slot_one.push_back(one ? 1 : 0);
        nodes += w;
    };
    for (int64_t r = 0; r < nr; ++r) {
        fv.clear();
        fc.clear();
        for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
            int32_t v = P->row_var[e];
            if (P->fixed[v] < 0) { fv.push_back(internal[v]); fc.push_back(P->row_coef[e]); }
        }
        const int n = int(fv.size());
        if (n == 0) continue;
        const int rr = res[r];
        int ptot = 0, qtot = 0;
        for (int8_t c : fc) (c > 0 ? ptot : qtot)++;
        lo.assign(n + 1, 0);
        wd.assign(n + 1, 0);
        int ppre = 0, qpre = 0;
        for (int l = 0; l <= n; ++l) {
            int lo_l = std::max(-qpre, rr - (ptot - ppre));
            int hi_l = std::min(ppre, rr + (qtot - qpre));
            lo[l] = lo_l;
            wd[l] = hi_l - lo_l + 1;
            if (wd[l] < 1 || wd[l] > kMaxWidth) {
                *err = wd[l] < 1 ? "empty BDD layer after presolve" : "BDD layer wider than 32 nodes";
                return wd[l] < 1 ? DISCO_ERR_INFEASIBLE : DISCO_ERR_INVALID_ARG;
            }
            if (l < n) (fc[l] > 0 ? ppre : qpre)++;
        }
        // balanced segment boundaries
        int nseg = (split_chunk > 0 && n > split_chunk) ? (n + split_chunk - 1) / split_chunk : 1;
        std::vector<int64_t> cut_aux(nseg + 1, -1);  // first aux id of the cut before segment s (width > 1)
        for (int s = 1; s < nseg; ++s) {
            int b = int(int64_t(s) * n / nseg);
            if (wd[b] > 1) {
                if (wd[b] + 1 > kMaxWidth) { *err = "split layer too wide"; return DISCO_ERR_INVALID_ARG; }
                cut_aux[s] = next_aux;
                next_aux += wd[b];
            }
        }
        for (int s = 0; s < nseg; ++s) {
            int b0 = int(int64_t(s) * n / nseg), b1 = int(int64_t(s + 1) * n / nseg);
            Segment sg{r, s, int64_t(P->slot_var.size()), 0, 0};
            // prefix chain: read the one-hot y_1..y_k, enter node j of layer b0
            if (s > 0 && wd[b0] > 1) {
                int k = wd[b0];
                for (int j = 1; j <= k; ++j) {
                    int32_t var = int32_t(-1 - (cut_aux[s] + j - 1));  // auxiliaries resolved below
                    if (j < k) add_slot(var, j, j + 1, 0, j, true);
                    else add_slot(var, k, k, -1, k - 1, true);
                    sg.max_width = std::max(sg.max_width, j);
                }
            }
            for (int l = b0; l < b1; ++l) {
                int d0 = lo[l] - lo[l + 1];
                add_slot(fv[l], wd[l], wd[l + 1], d0, d0 + fc[l], false);
                sg.max_width = std::max(sg.max_width, wd[l]);
            }
            // suffix chain: y_j = 1 iff the path leaves through node j of layer b1
            if (s + 1 < nseg && wd[b1] > 1) {
                int k = wd[b1];
                for (int j = 1; j <= k; ++j) {
                    int32_t var = int32_t(-1 - (cut_aux[s + 1] + j - 1));
                    int w = j == 1 ? k : k - j + 2;
                    int wn = j < k ? k - j + 1 : 1;
                    add_slot(var, w, wn, -1, k - j, true);
                    sg.max_width = std::max(sg.max_width, w);
                }
            }
            sg.n_layers = int32_t(int64_t(P->slot_var.size()) - sg.first_slot);
            max_layers = std::max(max_layers, sg.n_layers);
            max_width = std::max(max_width, sg.max_width);
            P->segs.push_back(sg);
        }
    }
    P->n_aux = next_aux;
    const int64_t nint = P->n_free + P->n_aux;
    if (nint >= (int64_t(1) << 31)) { *err = "too many variables"; return DISCO_ERR_INVALID_ARG; }
    for (int32_t& v : P->slot_var)
        if (v < 0) v = int32_t(P->n_free + (-1 - int64_t(v)));
    // degree and rank of every slot
    P->deg.assign(size_t(nint), 0);
    const size_t ns = P->slot_var.size();
    P->slot_desc.resize(ns);
    P->slot_lam0.resize(ns);
    P->slot_lam0_lo.resize(ns);
    std::vector<uint8_t> rank(ns);
    for (size_t i = 0; i < ns; ++i) {
        uint8_t& dg = P->deg[P->slot_var[i]];
        rank[i] = dg;
        if (++dg > 7) { *err = "variable in more than 7 BDDs"; return DISCO_ERR_INVALID_ARG; }
    }
    for (size_t i = 0; i < ns; ++i) {
        int32_t v = P->slot_var[i];
        int dg = P->deg[v];
        P->slot_desc[i] = pack_desc(slot_w[i], slot_wn[i], slot_d0[i], slot_d1[i], slot_one[i], rank[i], dg);
        const double l0 = v < P->n_free ? P->cost[P->free_orig[v]] / dg : 0.0;
        P->slot_lam0[i] = float(l0);
        P->slot_lam0_lo[i] = float(l0 - double(P->slot_lam0[i]));
    }
    P->n_nodes = nodes;
    P->max_layers = max_layers;
    P->max_width = max_width;
    P->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return DISCO_OK;
}

}  // namespace disco
