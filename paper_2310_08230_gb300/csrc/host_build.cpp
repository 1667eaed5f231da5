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
// normalised by the largest kept c_p; segments are balanced (cut at floor(s n / S)) with
// S = min(ceil(n / chunk), the segment cap): a one-hot chain carries cost information across
// one cut per half-pass, so very long rows stay in few segments.
//
// For a +-1 row with residual right-hand side r, the nodes of layer l are the partial sums
// sigma of the first l variables that are reachable from 0 and from which r is reachable:
// sigma in [max(-Q_pre, r - P_suf), min(P_pre, r + Q_suf)] (P / Q: counts of +1 / -1
// coefficients before / from layer l). Node s of a layer stands for sigma = lo + s.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/disco.h"
#include "plan.h"

namespace disco {

// ---- cache of large host blocks (declared in plan.h)
namespace {
constexpr size_t kCachedMin = size_t(1) << 20;
struct BlockCache {
    std::mutex mu;
    std::multimap<size_t, void*> free_blocks;  // size class -> block
    size_t held = 0, cap = 0;
    bool poison = false;  // fill every block with 0xA5 when handed out (tests)
    BlockCache() {
        const char* e = std::getenv("DISCO_HOST_CACHE_MB");
        cap = size_t(e ? std::strtoull(e, nullptr, 10) : 2048) << 20;
        poison = std::getenv("DISCO_HOST_CACHE_POISON") != nullptr;
    }
};
BlockCache& block_cache() {  // never destroyed: blocks may be freed during static destruction
    static BlockCache* c = new BlockCache();
    return *c;
}
size_t block_class(size_t b) {
    const int lg = 63 - __builtin_clzll(uint64_t(b));
    const size_t step = size_t(1) << (lg - 3);
    return (b + step - 1) & ~(step - 1);
}
}  // namespace

void* host_block_alloc(size_t bytes) {
    if (bytes < kCachedMin) return ::operator new(bytes);
    const size_t c = block_class(bytes);
    BlockCache& k = block_cache();
    void* p = nullptr;
    {
        std::lock_guard<std::mutex> g(k.mu);
        const auto it = k.free_blocks.find(c);
        if (it != k.free_blocks.end()) {
            p = it->second;
            k.free_blocks.erase(it);
            k.held -= c;
        }
    }
    if (!p) p = ::operator new(c);
    if (k.poison) std::memset(p, 0xA5, c);
    return p;
}

void host_block_free(void* p, size_t bytes) noexcept {
    if (!p) return;
    if (bytes < kCachedMin) {
        ::operator delete(p);
        return;
    }
    const size_t c = block_class(bytes);
    BlockCache& k = block_cache();
    {
        std::lock_guard<std::mutex> g(k.mu);
        if (k.held + c <= k.cap) {
            try {
                k.free_blocks.emplace(c, p);
                k.held += c;
                return;
            } catch (...) {
            }
        }
    }
    ::operator delete(p);
}

namespace {

// vertex sequence of a degenerate triangle over an edge (a < b): 0 -> a, 1 -> b
const int kEdgePattern[6][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

// The patterns p whose first symbol is `first` and whose second and third symbols are
// allowed: bit p of kPatternMask[first][b1][b2], where bit s of b1 (b2) says that symbol s
// may sit at the second (third) corner.
struct PatternMasks {
    uint8_t m[2][4][4];
    constexpr PatternMasks() : m{} {
        for (int f = 0; f < 2; ++f)
            for (int b1 = 0; b1 < 4; ++b1)
                for (int b2 = 0; b2 < 4; ++b2) {
                    uint8_t x = 0;
                    for (int p = 0; p < 6; ++p)
                        if (kEdgePattern[p][0] == f && ((b1 >> kEdgePattern[p][1]) & 1) && ((b2 >> kEdgePattern[p][2]) & 1))
                            x = uint8_t(x | (1u << p));
                    m[f][b1][b2] = x;
                }
    }
};
constexpr PatternMasks kPatternMask{};

// Compressed incidence list: the items of vertex v are item[ptr[v] .. ptr[v+1]).
template <class T>
struct Csr {
    std::vector<int32_t> ptr;
    std::vector<T> item;
    template <class F>
    void for_each(int v, F f) const {
        for (int32_t i = ptr[v]; i < ptr[v + 1]; ++i) f(item[i]);
    }
};

struct MeshTopo {
    int nv = 0, nt = 0;
    const int32_t* T = nullptr;
    std::vector<std::pair<int, int>> edges;  // sorted unique (a < b)
    Csr<std::pair<int, int>> tri_at;         // vertex -> (triangle, corner), ascending triangle
    Csr<int32_t> tri_at0;                    // vertex -> triangles having it as corner 0
    Csr<int32_t> edge_at;                    // vertex -> incident edges, ascending
};

template <class T, class Fill>
Csr<T> make_csr(int nv, int64_t nitems, Fill fill) {
    Csr<T> c;
    c.ptr.assign(size_t(nv) + 1, 0);
    fill([&](int v, const T&) { ++c.ptr[v + 1]; });
    for (int v = 0; v < nv; ++v) c.ptr[v + 1] += c.ptr[v];
    c.item.resize(size_t(nitems));
    std::vector<int32_t> pos(c.ptr.begin(), c.ptr.end() - 1);
    fill([&](int v, const T& x) { c.item[pos[v]++] = x; });
    return c;
}

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
    t->tri_at = make_csr<std::pair<int, int>>(m.nv, 3 * int64_t(m.nt), [&](auto add) {
        for (int f = 0; f < m.nt; ++f)
            for (int k = 0; k < 3; ++k) add(m.T[3 * f + k], std::pair<int, int>(f, k));
    });
    t->tri_at0 = make_csr<int32_t>(m.nv, m.nt, [&](auto add) {
        for (int f = 0; f < m.nt; ++f) add(m.T[3 * f], int32_t(f));
    });
    const int ne = int(t->edges.size());
    t->edge_at = make_csr<int32_t>(m.nv, 2 * int64_t(ne), [&](auto add) {
        for (int e = 0; e < ne; ++e) {
            add(t->edges[e].first, int32_t(e));
            add(t->edges[e].second, int32_t(e));
        }
    });
    return DISCO_OK;
}

struct Elems {  // matching elements, structure of arrays
    pod_vector<int32_t> m, n;  // 3 per element
    pod_vector<uint8_t> type;
    pod_vector<int32_t> xe, ye;
    void push(int m0, int m1, int m2, int n0, int n1, int n2, int ty, int x, int y) {
        m.push_back(m0); m.push_back(m1); m.push_back(m2);
        n.push_back(n0); n.push_back(n1); n.push_back(n2);
        type.push_back(uint8_t(ty));
        xe.push_back(x);
        ye.push_back(y);
    }
    size_t size() const { return type.size(); }
    // k more elements of type ty, X element x; returns the first one's index
    size_t grow(size_t k, int ty, int x) {
        const size_t b = size();
        m.resize(3 * (b + k));
        n.resize(3 * (b + k));
        type.resize(b + k, uint8_t(ty));
        xe.resize(b + k, x);
        ye.resize(b + k);
        return b;
    }
};

// Sorts distinct codes in [0, range) ascending. Unless they are very sparse in their range, one pass
// over a bit set (`bits`: range / 64 zero words, left zero) replaces the comparison sort.
template <class T>
void sort_codes(std::vector<T>* c, int64_t range, std::vector<uint64_t>* bits) {
    const size_t k = c->size();
    const int64_t words = (range + 63) / 64;
    if (k < 16 || int64_t(k) * 32 < words) {  // a sort costs about k log k branchy steps
        std::sort(c->begin(), c->end());
        return;
    }
    if (int64_t(bits->size()) < words) bits->assign(size_t(words), 0);
    uint64_t* b = bits->data();
    for (const T x : *c) b[x >> 6] |= uint64_t(1) << (x & 63);
    size_t o = 0;
    for (int64_t w = 0; w < words && o < k; ++w)
        for (uint64_t x = b[w]; x; x &= x - 1) (*c)[o++] = T(w * 64 + __builtin_ctzll(x));
    for (const T x : *c) b[x >> 6] = 0;
}


// Candidate pairs: a bit row per X vertex (cache resident) and the allowed Y vertices of
// every X vertex in ascending order.
struct Allowed {
    bool full = true;
    int words = 0;
    std::vector<uint64_t> bits;
    Csr<int32_t> row;
    bool operator()(int a, int b) const {
        return full || ((bits[size_t(a) * words + (b >> 6)] >> (b & 63)) & 1u);
    }
};

// Runs body(lo, hi, out) over [0, n) in contiguous chunks on up to `threads` threads and
// concatenates the per-chunk outputs in order (the result does not depend on threads).
// Runs the element generators of all five types over contiguous index chunks on one pool of
// threads and concatenates the chunk outputs in (type, chunk) order, i.e. canonical order
// whatever the thread count.
struct Job {
    int type, lo, hi;
};

template <class Gen>
void run_jobs(const std::vector<Job>& jobs, int threads, Elems* out, Gen gen) {
    const int nj = int(jobs.size());
    std::vector<Elems> parts(nj);
    auto run = [&](auto&& job) { parallel_tasks(nj, threads, [&](int64_t c) { job(int(c)); }); };
    run([&](int c) { gen(jobs[c], &parts[c]); });
    std::vector<size_t> off(nj + 1, out->size());
    for (int c = 0; c < nj; ++c) off[c + 1] = off[c] + parts[c].size();
    const size_t total = off[nj];
    out->m.resize(3 * total);
    out->n.resize(3 * total);
    out->type.resize(total);
    out->xe.resize(total);
    out->ye.resize(total);
    run([&](int c) {
        const Elems& q = parts[c];
        const size_t o = off[c];
        std::copy(q.m.begin(), q.m.end(), out->m.begin() + 3 * o);
        std::copy(q.n.begin(), q.n.end(), out->n.begin() + 3 * o);
        std::copy(q.type.begin(), q.type.end(), out->type.begin() + o);
        std::copy(q.xe.begin(), q.xe.end(), out->xe.begin() + o);
        std::copy(q.ye.begin(), q.ye.end(), out->ye.begin() + o);
        Elems().m.swap(parts[c].m);
    });
}

void enumerate(const MeshTopo& X, const MeshTopo& Y, const Allowed& A, int threads, Elems* out) {
    const int32_t* TX = X.T;
    const int32_t* TY = Y.T;
    const int count[5] = {X.nt, X.nt, int(X.edges.size()), X.nt, X.nv};
    std::vector<Job> jobs;
    for (int ty = 0; ty < 5; ++ty) {
        const int nch = std::max(1, std::min(threads * 4, count[ty] / 16 + 1));
        for (int c = 0; c < nch; ++c)
            jobs.push_back(Job{ty, int(int64_t(count[ty]) * c / nch), int(int64_t(count[ty]) * (c + 1) / nch)});
    }
    run_jobs(jobs, threads, out, [&](const Job& j, Elems* o) {
        const int lo = j.lo, hi = j.hi;
        std::vector<uint64_t> bits;  // sort_codes' bit set
        switch (j.type) {
            case 0: {  // type 0: X triangle t, Y triangle s, rotation r: corner v -> (t_v, s_{(v+r)%3})
            std::vector<int64_t> cand;
            for (int t = lo; t < hi; ++t) {
                int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
                cand.clear();
                A.row.for_each(m0, [&](int n0) {
                    Y.tri_at.for_each(n0, [&](std::pair<int, int> sr) {
                        const int s = sr.first, r = sr.second;
                        if (A(m1, TY[3 * s + (r + 1) % 3]) && A(m2, TY[3 * s + (r + 2) % 3])) cand.push_back(int64_t(s) * 3 + r);
                    });
                });
                sort_codes(&cand, int64_t(Y.nt) * 3, &bits);
                const size_t b = o->grow(cand.size(), 0, t);
                int32_t* om = o->m.data() + 3 * b;
                int32_t* on = o->n.data() + 3 * b;
                int32_t* oy = o->ye.data() + b;
                for (const int64_t c : cand) {
                    const int s = int(c / 3), r = int(c % 3);
                    om[0] = m0; om[1] = m1; om[2] = m2;
                    on[0] = TY[3 * s + r]; on[1] = TY[3 * s + (r + 1) % 3]; on[2] = TY[3 * s + (r + 2) % 3];
                    *oy++ = s;
                    om += 3;
                    on += 3;
                }
            }
                break;
            }
            case 1: {  // type 1: X triangle t, Y edge e = (a < b), pattern p: corner v -> (t_v, pattern symbol)
            // per edge at n0 the four candidate bits (m1, a), (m1, b), (m2, a), (m2, b) decide
            // the three patterns that start at n0
            std::vector<int64_t> cand;
            for (int t = lo; t < hi; ++t) {
                int m[3] = {TX[3 * t], TX[3 * t + 1], TX[3 * t + 2]};
                cand.clear();
                A.row.for_each(m[0], [&](int n0) {
                    Y.edge_at.for_each(n0, [&](int e) {
                        const int ab[2] = {Y.edges[e].first, Y.edges[e].second};
                        const int role = ab[0] == n0 ? 0 : 1;  // patterns whose first corner is n0
                        const int b1 = int(A(m[1], ab[0])) | int(A(m[1], ab[1])) << 1;
                        const int b2 = int(A(m[2], ab[0])) | int(A(m[2], ab[1])) << 1;
                        for (unsigned x = kPatternMask.m[role][b1][b2]; x; x &= x - 1)
                            cand.push_back(int64_t(e) * 6 + __builtin_ctz(x));
                    });
                });
                sort_codes(&cand, int64_t(Y.edges.size()) * 6, &bits);
                const size_t b = o->grow(cand.size(), 1, t);
                int32_t* om = o->m.data() + 3 * b;
                int32_t* on = o->n.data() + 3 * b;
                int32_t* oy = o->ye.data() + b;
                for (const int64_t c : cand) {
                    const int e = int(c / 6), p = int(c % 6);
                    const int ab[2] = {Y.edges[e].first, Y.edges[e].second};
                    om[0] = m[0]; om[1] = m[1]; om[2] = m[2];
                    on[0] = ab[kEdgePattern[p][0]]; on[1] = ab[kEdgePattern[p][1]]; on[2] = ab[kEdgePattern[p][2]];
                    *oy++ = e;
                    om += 3;
                    on += 3;
                }
            }
                break;
            }
            case 2: {  // type 2: X edge e = (a < b), Y triangle s, pattern p: corner v -> (pattern symbol, s_v)
            // one walk over the candidate row of each end x0 of the edge; per Y triangle s at a
            // candidate n0 = s_0 the four bits (a, s_1), (b, s_1), (a, s_2), (b, s_2) decide the
            // three patterns that start with x0
            std::vector<int64_t> cand;
            for (int e = lo; e < hi; ++e) {
                const int ab[2] = {X.edges[e].first, X.edges[e].second};
                cand.clear();
                for (int first = 0; first < 2; ++first) {
                    A.row.for_each(ab[first], [&](int n0) {
                        Y.tri_at0.for_each(n0, [&](int s) {
                            const int s1 = TY[3 * s + 1], s2 = TY[3 * s + 2];
                            const int b1 = int(A(ab[0], s1)) | int(A(ab[1], s1)) << 1;
                            const int b2 = int(A(ab[0], s2)) | int(A(ab[1], s2)) << 1;
                            for (unsigned x = kPatternMask.m[first][b1][b2]; x; x &= x - 1)
                                cand.push_back(int64_t(s) * 6 + __builtin_ctz(x));
                        });
                    });
                }
                sort_codes(&cand, int64_t(Y.nt) * 6, &bits);
                const size_t b = o->grow(cand.size(), 2, e);
                int32_t* om = o->m.data() + 3 * b;
                int32_t* on = o->n.data() + 3 * b;
                int32_t* oy = o->ye.data() + b;
                for (const int64_t c : cand) {
                    const int s = int(c / 6), p = int(c % 6);
                    om[0] = ab[kEdgePattern[p][0]]; om[1] = ab[kEdgePattern[p][1]]; om[2] = ab[kEdgePattern[p][2]];
                    on[0] = TY[3 * s]; on[1] = TY[3 * s + 1]; on[2] = TY[3 * s + 2];
                    *oy++ = s;
                    om += 3;
                    on += 3;
                }
            }
                break;
            }
            case 3: {  // type 3: X triangle t, Y vertex n
            for (int t = lo; t < hi; ++t) {
                int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
                A.row.for_each(m0, [&](int n) {
                    if (A(m1, n) && A(m2, n)) o->push(m0, m1, m2, n, n, n, 3, t, n);
                });
            }
                break;
            }
            case 4: {  // type 4: X vertex m, Y triangle s
            std::vector<int> cand;
            for (int mv = lo; mv < hi; ++mv) {
                cand.clear();
                A.row.for_each(mv, [&](int n0) {
                    Y.tri_at0.for_each(n0, [&](int s) {
                        if (A(mv, TY[3 * s + 1]) && A(mv, TY[3 * s + 2])) cand.push_back(s);
                    });
                });
                sort_codes(&cand, int64_t(Y.nt), &bits);
                const size_t b = o->grow(cand.size(), 4, mv);
                int32_t* om = o->m.data() + 3 * b;
                int32_t* on = o->n.data() + 3 * b;
                int32_t* oy = o->ye.data() + b;
                for (const int s : cand) {
                    om[0] = mv; om[1] = mv; om[2] = mv;
                    on[0] = TY[3 * s]; on[1] = TY[3 * s + 1]; on[2] = TY[3 * s + 2];
                    *oy++ = s;
                    om += 3;
                    on += 3;
                }
            }
                break;
            }
        }
    });
}

// The same product space by bit-set algebra, for candidate masks that are dense enough: per X
// vertex m, TB[m][c] has bit s set iff (m, corner c of Y triangle s) is allowed, and EB[m][j]
// bit e iff (m, end j of Y edge e) is allowed (built from the candidate rows, 12 bits per
// candidate on average). An element is allowed iff its three corner pairs are, so each type
// is the AND of three such rows, one word at a time, and reading the set bits in ascending
// order per word, then rotation or pattern ascending, gives the canonical order that the
// sorted codes of enumerate() give.
bool dense_enumeration(const MeshTopo& X, const MeshTopo& Y, const Allowed& A) {
    if (const char* e = std::getenv("DISCO_HOST_ENUM")) return std::strcmp(e, "sparse") != 0 && !A.full;
    if (A.full) return false;
    const double wt = double((Y.nt + 63) / 64), we = double((int64_t(Y.edges.size()) + 63) / 64);
    if (double(X.nv) * (3 * wt + 2 * we) * 8.0 > double(int64_t(1) << 30)) return false;  // bit sets above 1 GB
    const double dense = double(X.nt) * (9 * wt + 18 * we + 3 * A.words) + double(X.edges.size()) * 18 * wt +
                         double(X.nv) * 3 * wt;
    const double cand = double(A.row.ptr[size_t(X.nv)]) / double(std::max(1, X.nv));
    const double sparse = cand * (12.0 * X.nt + 24.0 * double(X.edges.size()) + 6.0 * X.nv);
    return dense < 4.0 * sparse;  // a word AND is far cheaper than a random bit lookup and branch
}

void enumerate_dense(const MeshTopo& X, const MeshTopo& Y, const Allowed& A, int threads, Elems* out) {
    const int32_t* TX = X.T;
    const int32_t* TY = Y.T;
    const int64_t WT = (Y.nt + 63) / 64, WE = (int64_t(Y.edges.size()) + 63) / 64, WV = A.words;
    pod_vector<uint64_t> TB(static_cast<size_t>(int64_t(X.nv) * 3 * WT)), EB(static_cast<size_t>(int64_t(X.nv) * 2 * WE));
    parallel_chunks(X.nv, threads, [&](int, int64_t lo, int64_t hi) {
        for (int64_t m = lo; m < hi; ++m) {
            uint64_t* tb = TB.data() + m * 3 * WT;
            uint64_t* eb = EB.data() + m * 2 * WE;
            std::fill(tb, tb + 3 * WT, uint64_t(0));
            std::fill(eb, eb + 2 * WE, uint64_t(0));
            A.row.for_each(int(m), [&](int n) {
                Y.tri_at.for_each(n, [&](std::pair<int, int> sc) {
                    tb[sc.second * WT + (sc.first >> 6)] |= uint64_t(1) << (sc.first & 63);
                });
                Y.edge_at.for_each(n, [&](int e) {
                    eb[(Y.edges[size_t(e)].first == n ? 0 : 1) * WE + (e >> 6)] |= uint64_t(1) << (e & 63);
                });
            });
        }
    });
    auto tb_row = [&](int m, int c) { return TB.data() + (int64_t(m) * 3 + c) * WT; };
    auto eb_row = [&](int m, int j) { return EB.data() + (int64_t(m) * 2 + j) * WE; };
    const int count[5] = {X.nt, X.nt, int(X.edges.size()), X.nt, X.nv};
    std::vector<Job> jobs;
    for (int ty = 0; ty < 5; ++ty) {
        const int nch = std::max(1, std::min(threads * 4, count[ty] / 16 + 1));
        for (int c = 0; c < nch; ++c)
            jobs.push_back(Job{ty, int(int64_t(count[ty]) * c / nch), int(int64_t(count[ty]) * (c + 1) / nch)});
    }
    run_jobs(jobs, threads, out, [&](const Job& j, Elems* o) {
        std::vector<uint64_t> x;  // the AND words of each rotation / pattern of one X element
        // K rows of W words in x: the elements in (bit, row) order, handed to emit(row, bit index)
        auto for_bits = [&](int K, int64_t W, auto&& emit) {
            for (int64_t w = 0; w < W; ++w) {
                uint64_t u = 0;
                for (int r = 0; r < K; ++r) u |= x[size_t(r * W + w)];
                for (; u; u &= u - 1) {
                    const int b = __builtin_ctzll(u);
                    for (int r = 0; r < K; ++r)
                        if ((x[size_t(r * W + w)] >> b) & 1u) emit(r, int(w * 64 + b));
                }
            }
        };
        auto and3 = [&](int r, int64_t W, const uint64_t* p, const uint64_t* q, const uint64_t* u) {
            size_t k = 0;
            uint64_t* d = x.data() + r * W;
            for (int64_t w = 0; w < W; ++w) {
                d[w] = p[w] & q[w] & u[w];
                k += size_t(__builtin_popcountll(d[w]));
            }
            return k;
        };
        switch (j.type) {
            case 0: {  // X triangle t, Y triangle s, rotation r: corner v -> (t_v, s_{(v+r)%3})
                x.resize(size_t(3 * WT));
                for (int t = j.lo; t < j.hi; ++t) {
                    const int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
                    size_t k = 0;
                    for (int r = 0; r < 3; ++r)
                        k += and3(r, WT, tb_row(m0, r), tb_row(m1, (r + 1) % 3), tb_row(m2, (r + 2) % 3));
                    const size_t b = o->grow(k, 0, t);
                    int32_t* om = o->m.data() + 3 * b;
                    int32_t* on = o->n.data() + 3 * b;
                    int32_t* oy = o->ye.data() + b;
                    for_bits(3, WT, [&](int r, int s) {
                        om[0] = m0; om[1] = m1; om[2] = m2;
                        on[0] = TY[3 * s + r]; on[1] = TY[3 * s + (r + 1) % 3]; on[2] = TY[3 * s + (r + 2) % 3];
                        *oy++ = s;
                        om += 3;
                        on += 3;
                    });
                }
                break;
            }
            case 1: {  // X triangle t, Y edge e = (a < b), pattern p: corner v -> (t_v, pattern symbol v)
                x.resize(size_t(6 * WE));
                for (int t = j.lo; t < j.hi; ++t) {
                    const int m[3] = {TX[3 * t], TX[3 * t + 1], TX[3 * t + 2]};
                    size_t k = 0;
                    for (int p = 0; p < 6; ++p)
                        k += and3(p, WE, eb_row(m[0], kEdgePattern[p][0]), eb_row(m[1], kEdgePattern[p][1]),
                                  eb_row(m[2], kEdgePattern[p][2]));
                    const size_t b = o->grow(k, 1, t);
                    int32_t* om = o->m.data() + 3 * b;
                    int32_t* on = o->n.data() + 3 * b;
                    int32_t* oy = o->ye.data() + b;
                    for_bits(6, WE, [&](int p, int e) {
                        const int ab[2] = {Y.edges[size_t(e)].first, Y.edges[size_t(e)].second};
                        om[0] = m[0]; om[1] = m[1]; om[2] = m[2];
                        on[0] = ab[kEdgePattern[p][0]]; on[1] = ab[kEdgePattern[p][1]]; on[2] = ab[kEdgePattern[p][2]];
                        *oy++ = e;
                        om += 3;
                        on += 3;
                    });
                }
                break;
            }
            case 2: {  // X edge e = (a < b), Y triangle s, pattern p: corner v -> (pattern symbol v, s_v)
                x.resize(size_t(6 * WT));
                for (int e = j.lo; e < j.hi; ++e) {
                    const int ab[2] = {X.edges[size_t(e)].first, X.edges[size_t(e)].second};
                    size_t k = 0;
                    for (int p = 0; p < 6; ++p)
                        k += and3(p, WT, tb_row(ab[kEdgePattern[p][0]], 0), tb_row(ab[kEdgePattern[p][1]], 1),
                                  tb_row(ab[kEdgePattern[p][2]], 2));
                    const size_t b = o->grow(k, 2, e);
                    int32_t* om = o->m.data() + 3 * b;
                    int32_t* on = o->n.data() + 3 * b;
                    int32_t* oy = o->ye.data() + b;
                    for_bits(6, WT, [&](int p, int s) {
                        om[0] = ab[kEdgePattern[p][0]]; om[1] = ab[kEdgePattern[p][1]]; om[2] = ab[kEdgePattern[p][2]];
                        on[0] = TY[3 * s]; on[1] = TY[3 * s + 1]; on[2] = TY[3 * s + 2];
                        *oy++ = s;
                        om += 3;
                        on += 3;
                    });
                }
                break;
            }
            case 3: {  // X triangle t, Y vertex n
                x.resize(size_t(WV));
                for (int t = j.lo; t < j.hi; ++t) {
                    const int m0 = TX[3 * t], m1 = TX[3 * t + 1], m2 = TX[3 * t + 2];
                    const size_t k = and3(0, WV, A.bits.data() + size_t(m0) * WV, A.bits.data() + size_t(m1) * WV,
                                          A.bits.data() + size_t(m2) * WV);
                    const size_t b = o->grow(k, 3, t);
                    int32_t* om = o->m.data() + 3 * b;
                    int32_t* on = o->n.data() + 3 * b;
                    int32_t* oy = o->ye.data() + b;
                    for_bits(1, WV, [&](int, int n) {
                        om[0] = m0; om[1] = m1; om[2] = m2;
                        on[0] = n; on[1] = n; on[2] = n;
                        *oy++ = n;
                        om += 3;
                        on += 3;
                    });
                }
                break;
            }
            case 4: {  // X vertex m, Y triangle s
                x.resize(size_t(WT));
                for (int mv = j.lo; mv < j.hi; ++mv) {
                    const size_t k = and3(0, WT, tb_row(mv, 0), tb_row(mv, 1), tb_row(mv, 2));
                    const size_t b = o->grow(k, 4, mv);
                    int32_t* om = o->m.data() + 3 * b;
                    int32_t* on = o->n.data() + 3 * b;
                    int32_t* oy = o->ye.data() + b;
                    for_bits(1, WT, [&](int, int s) {
                        om[0] = mv; om[1] = mv; om[2] = mv;
                        on[0] = TY[3 * s]; on[1] = TY[3 * s + 1]; on[2] = TY[3 * s + 2];
                        *oy++ = s;
                        om += 3;
                        on += 3;
                    });
                }
                break;
            }
        }
    });
}

// One boundary edge of one element: its smaller product vertex (m, n) is implied by the
// bucket (m) and `lo_n`; `hi` is the larger product vertex m' * nvy + n'; `id` packs the
// entry 3 * element + corner and the direction bit.
struct EdgeEntry {
    uint32_t lo_n;
    uint32_t hi;
    uint32_t id;
    bool operator<(const EdgeEntry& o) const {
        return lo_n != o.lo_n ? lo_n < o.lo_n : (hi != o.hi ? hi < o.hi : id < o.id);
    }
    bool same_edge(const EdgeEntry& o) const { return lo_n == o.lo_n && hi == o.hi; }
};

// BDD segments of a contiguous range of rows, with auxiliary ids local to the range.
struct RowChunk {
    pod_vector<int32_t> var;    // internal variable id; auxiliaries as -1 - local index
    pod_vector<uint32_t> desc;  // packed layer descriptor (pack_desc)
    std::vector<Segment> segs;  // first_slot local to the chunk
    int64_t n_aux = 0, nodes = 0;
    int max_layers = 0, max_width = 0;
    std::string err;
    int rc = 0;
};

}  // namespace

void mixed_areas(const MeshIn& M, std::vector<double>* out) {
    out->assign(size_t(M.nv), 0.0);
    for (int t = 0; t < M.nt; ++t) {
        const int id[3] = {M.T[3 * t], M.T[3 * t + 1], M.T[3 * t + 2]};
        double p[3][3];
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) p[v][k] = double(M.V[3 * size_t(id[v]) + k]);
        // edge vectors and the corner dot products: corner v between edges to v+1 and v+2
        auto sub = [](const double* a, const double* b, double* r) {
            for (int k = 0; k < 3; ++k) r[k] = a[k] - b[k];
        };
        auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
        double e[3][2][3], dv[3], len2[3];
        for (int v = 0; v < 3; ++v) {
            sub(p[(v + 1) % 3], p[v], e[v][0]);
            sub(p[(v + 2) % 3], p[v], e[v][1]);
            dv[v] = dot(e[v][0], e[v][1]);
        }
        double cr[3];
        cr[0] = e[0][0][1] * e[0][1][2] - e[0][0][2] * e[0][1][1];
        cr[1] = e[0][0][2] * e[0][1][0] - e[0][0][0] * e[0][1][2];
        cr[2] = e[0][0][0] * e[0][1][1] - e[0][0][1] * e[0][1][0];
        const double twice = std::sqrt(dot(cr, cr));  // twice the triangle area
        if (twice <= 0.0) continue;
        for (int v = 0; v < 3; ++v) len2[v] = dot(e[v][0], e[v][0]);  // |p_v p_{v+1}|^2
        int obtuse = -1;
        for (int v = 0; v < 3; ++v)
            if (dv[v] < 0.0) obtuse = v;
        if (obtuse < 0) {
            // cot of the angle at corner v = dot / (2 area); Voronoi part of corner v uses the
            // two edges at v and the cotangents of the opposite angles
            for (int v = 0; v < 3; ++v) {
                const int a = (v + 1) % 3, b = (v + 2) % 3;
                const double cot_a = dv[a] / twice, cot_b = dv[b] / twice;
                // |v b|^2 cot(angle at a) + |v a|^2 cot(angle at b)
                (*out)[id[v]] += (len2[b] * cot_a + len2[v] * cot_b) / 8.0;
            }
        } else {
            for (int v = 0; v < 3; ++v) (*out)[id[v]] += (v == obtuse ? 0.25 : 0.125) * twice;
        }
    }
}

int build_plan(const MeshIn& Xin, const MeshIn& Yin, const float* d, const uint8_t* mask, int split_chunk,
               int split_max_segments, int threads, Plan* P, std::string* err, bool normalize, int cost_model) {
    auto t0 = std::chrono::steady_clock::now();
    Trace tr;
    if (threads <= 0) threads = std::max(1u, std::thread::hardware_concurrency());
    MeshTopo X, Y;
    int chiX = 0, chiY = 0;
    std::string errXY[2];
    int rcXY[2] = {DISCO_OK, DISCO_OK};
    parallel_tasks(2, threads, [&](int64_t k) {
        rcXY[k] = k == 0 ? topo(Xin, &X, &chiX, &errXY[0]) : topo(Yin, &Y, &chiY, &errXY[1]);
    });
    if (rcXY[0]) { *err = "mesh X: " + errXY[0]; return rcXY[0]; }
    if (rcXY[1]) { *err = "mesh Y: " + errXY[1]; return rcXY[1]; }
    if (chiX != chiY) { *err = "Euler characteristics differ"; return DISCO_ERR_GENUS_MISMATCH; }
    const int nvx = X.nv, nvy = Y.nv;
    P->nvx = nvx;
    P->nvy = nvy;

    tr.mark("meshes");
    // ---- candidate rows
    Allowed A;
    A.full = mask == nullptr;
    A.words = (nvy + 63) / 64;
    A.row.ptr.assign(size_t(nvx) + 1, 0);
    if (!A.full) {
        A.bits.assign(size_t(nvx) * A.words, 0);
        parallel_chunks(nvx, threads, [&](int, int64_t lo, int64_t hi) {
            for (int64_t m = lo; m < hi; ++m) {
                int32_t c = 0;
                for (int n = 0; n < nvy; ++n)
                    if (mask[size_t(m) * nvy + n]) {
                        A.bits[size_t(m) * A.words + (n >> 6)] |= uint64_t(1) << (n & 63);
                        ++c;
                    }
                A.row.ptr[m + 1] = c;
            }
        });
    } else {
        for (int m = 0; m < nvx; ++m) A.row.ptr[m + 1] = nvy;
    }
    for (int m = 0; m < nvx; ++m) A.row.ptr[m + 1] += A.row.ptr[m];
    A.row.item.resize(size_t(A.row.ptr[nvx]));
    parallel_chunks(nvx, threads, [&](int, int64_t lo, int64_t hi) {
        for (int64_t m = lo; m < hi; ++m) {
            int32_t o = A.row.ptr[m];
            for (int n = 0; n < nvy; ++n)
                if (A(int(m), n)) A.row.item[o++] = n;
        }
    });

    tr.mark("candidate rows");
    // ---- product space
    Elems E;
    if (dense_enumeration(X, Y, A))
        enumerate_dense(X, Y, A, threads, &E);
    else
        enumerate(X, Y, A, threads, &E);
    const int64_t nv = int64_t(E.size());
    if (nv == 0) { *err = "empty product space"; return DISCO_ERR_INFEASIBLE; }
    if (nv >= (int64_t(1) << 31)) { *err = "product space too large"; return DISCO_ERR_INVALID_ARG; }
    P->nvars = nv;
    P->vm = std::move(E.m);
    P->vn = std::move(E.n);

    tr.mark("product space");
    // ---- costs: mean of the three pair costs (or Eq. 2), normalised by the largest
    const int nth = threads;
    std::vector<double> aX, aY;
    if (cost_model == 1) {
        if (!Xin.V || !Yin.V) { *err = "cost model 1 needs vertex positions"; return DISCO_ERR_INVALID_ARG; }
        mixed_areas(Xin, &aX);
        mixed_areas(Yin, &aY);
    }
    P->cost.resize(nv);
    {
        std::vector<double> cmaxs(nth, 0.0);
        std::vector<int> bad(nth, 0);
        parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
            double mx = 0.0;  // per-chunk results are written once (no false sharing)
            int nonfinite = 0;
            for (int64_t i = lo; i < hi; ++i) {
                double x = 0.0;
                if (cost_model == 1) {
                    for (int v = 0; v < 3; ++v) {
                        const int m = P->vm[3 * i + v], nn = P->vn[3 * i + v];
                        x += (aX[m] + aY[nn]) * double(d[size_t(m) * nvy + nn]);
                    }
                } else {
                    for (int v = 0; v < 3; ++v) x += double(d[size_t(P->vm[3 * i + v]) * nvy + P->vn[3 * i + v]]);
                    x /= 3.0;
                }
                if (!(x >= 0.0) || x > 3.0e38) nonfinite = 1;
                P->cost[i] = x;
                mx = std::max(mx, x);
            }
            cmaxs[c] = mx;
            bad[c] = nonfinite;
        });
        for (int c = 0; c < nth; ++c)
            if (bad[c]) { *err = "pair costs must be finite and >= 0"; return DISCO_ERR_INVALID_ARG; }
        const double cmax = *std::max_element(cmaxs.begin(), cmaxs.end());
        P->cost_scale = 1.0;
        P->cost_scale_elem = -1;
        P->cost_max = cmax;
        if (normalize && cmax > 0) {
            P->cost_max = 1.0;  // x / cmax is at most 1, and exactly 1 for the largest
            P->cost_scale = cmax;
            for (int64_t i = 0; i < nv; ++i)
                if (P->cost[i] == cmax) { P->cost_scale_elem = i; break; }
            parallel_chunks(nv, nth, [&](int, int64_t lo, int64_t hi) {
                for (int64_t i = lo; i < hi; ++i) P->cost[i] /= cmax;
            });
        }
    }

    if (cost_model == 1) {  // kept for the chain rule of the gradient
        P->area_x = std::move(aX);
        P->area_y = std::move(aY);
    }
    tr.mark("costs");
    // ---- closedness rows: product edge (p, q), p < q in (m, n) order. Entries are bucketed by
    // the X vertex of p, each bucket sorted by (key, entry), rows are the runs of equal keys.
    if (uint64_t(nvx) * uint64_t(nvy) >= (uint64_t(1) << 32)) { *err = "meshes too large"; return DISCO_ERR_INVALID_ARG; }
    const int64_t ne = 3 * nv;
    if (ne >= (int64_t(1) << 31)) { *err = "product space too large"; return DISCO_ERR_INVALID_ARG; }
    pod_vector<EdgeEntry> ent(static_cast<size_t>(ne));
    std::vector<int64_t> bstart(size_t(nvx) + 1, 0);
    {
        // corner v of element i and corner v+1: (m, n) pairs, ordered lexicographically
        auto edge_of = [&](int64_t i, int v, int* lm, EdgeEntry* out) {
            const int w = (v + 1) % 3;
            const int ma = P->vm[3 * i + v], na = P->vn[3 * i + v];
            const int mb = P->vm[3 * i + w], nb = P->vn[3 * i + w];
            const bool fwd = ma < mb || (ma == mb && na < nb);
            *lm = fwd ? ma : mb;
            out->lo_n = uint32_t(fwd ? na : nb);
            out->hi = fwd ? uint32_t(mb) * uint32_t(nvy) + uint32_t(nb) : uint32_t(ma) * uint32_t(nvy) + uint32_t(na);
            out->id = uint32_t(3 * i + v) * 2u + (fwd ? 0u : 1u);
        };
        std::vector<std::vector<int64_t>> cnt(nth, std::vector<int64_t>(size_t(nvx), 0));
        parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i)
                for (int v = 0; v < 3; ++v) {
                    int lm;
                    EdgeEntry x;
                    edge_of(i, v, &lm, &x);
                    ++cnt[c][lm];
                }
        });
        // bucket offsets per (bucket, chunk) in chunk order: entries keep their id order per bucket
        std::vector<std::vector<int64_t>> off(nth, std::vector<int64_t>(size_t(nvx), 0));
        int64_t run = 0;
        for (int m = 0; m < nvx; ++m) {
            bstart[m] = run;
            for (int c = 0; c < nth; ++c) {
                off[c][m] = run;
                run += cnt[c][m];
            }
        }
        bstart[nvx] = run;
        parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i)
                for (int v = 0; v < 3; ++v) {
                    int lm;
                    EdgeEntry x;
                    edge_of(i, v, &lm, &x);
                    ent[off[c][lm]++] = x;
                }
        });
    }
    tr.mark("closedness buckets");
    // order each bucket by (smaller vertex, larger vertex, entry); count rows per bucket.
    // Entries arrive in entry order. The smaller product vertex (m, n) of an edge is a corner
    // of an element, so n is a candidate of m: a stable counting sort on n's position in the
    // candidate row of m, then a stable sort by the larger vertex inside each group.
    std::vector<int64_t> brows(size_t(nvx) + 1, 0);
    // The larger vertex (m', n') of an edge in bucket m has m' in the closed 1-ring of m (the
    // edge joins two corners of one element), so the counting key is (position of n in m's
    // candidate row, rank of m' in m's sorted closed ring); inside a key group only n' is left
    // to order (a few entries). Any entry outside these sets falls back to a plain sort.
    const int nbc = std::max(1, std::min(nth * 16, nvx));  // bucket ranges, taken dynamically
    parallel_tasks(nbc, nth, [&](int64_t c) {
        std::vector<int32_t> pos_of(static_cast<size_t>(nvy), -1);
        std::vector<int32_t> rank_of(static_cast<size_t>(nvx), -1);
        std::vector<int32_t> ring;
        std::vector<int64_t> cnt, cnt2;
        std::vector<int32_t> key, key2, ny;
        std::vector<EdgeEntry> tmp;
        {
            for (int64_t m = int64_t(nvx) * c / nbc; m < int64_t(nvx) * (c + 1) / nbc; ++m) {
                const int64_t b0 = bstart[m], b1 = bstart[m + 1], nb = b1 - b0;
                const int32_t* cand = A.row.item.data() + A.row.ptr[m];
                const int ncand = A.row.ptr[m + 1] - A.row.ptr[m];
                for (int i = 0; i < ncand; ++i) pos_of[cand[i]] = i;
                ring.assign(1, int32_t(m));
                X.edge_at.for_each(int(m), [&](int e) {
                    ring.push_back(X.edges[e].first == m ? X.edges[e].second : X.edges[e].first);
                });
                std::sort(ring.begin(), ring.end());
                const int R = int(ring.size());
                for (int i = 0; i < R; ++i) rank_of[ring[i]] = i;
                key.resize(size_t(nb));
                ny.resize(size_t(nb));
                bool ok = true;
                for (int64_t e = b0; e < b1 && ok; ++e) {
                    const int32_t p = pos_of[ent[e].lo_n];
                    const int32_t mh = int32_t(ent[e].hi / uint32_t(nvy));
                    const int32_t q = rank_of[mh];
                    ok = p >= 0 && p < ncand && cand[p] == int32_t(ent[e].lo_n) && q >= 0 && q < R && ring[q] == mh;
                    key[e - b0] = p * R + q;
                    ny[e - b0] = int32_t(ent[e].hi - uint32_t(mh) * uint32_t(nvy));  // n' of the larger vertex
                }
                if (!ok) {
                    std::sort(ent.data() + b0, ent.data() + b1);
                } else {
                    // two stable counting sorts: by n' (inside a key group, hi orders by n'),
                    // then by the key; entries of one product edge keep their entry order
                    const int nk = ncand * R;
                    cnt2.assign(size_t(nvy) + 1, 0);
                    for (int64_t e = 0; e < nb; ++e) ++cnt2[size_t(ny[e]) + 1];
                    for (int i = 0; i < nvy; ++i) cnt2[i + 1] += cnt2[i];
                    tmp.resize(size_t(nb));
                    key2.resize(size_t(nb));
                    for (int64_t e = 0; e < nb; ++e) {
                        const int64_t o = cnt2[size_t(ny[e])]++;
                        tmp[size_t(o)] = ent[b0 + e];
                        key2[size_t(o)] = key[e];
                    }
                    cnt.assign(size_t(nk) + 1, 0);
                    for (int64_t e = 0; e < nb; ++e) ++cnt[size_t(key2[e]) + 1];
                    for (int i = 0; i < nk; ++i) cnt[i + 1] += cnt[i];
                    for (int64_t e = 0; e < nb; ++e) ent[b0 + cnt[size_t(key2[e])]++] = tmp[size_t(e)];
                }
                for (int i = 0; i < R; ++i) rank_of[ring[i]] = -1;
                int64_t r = 0;
                for (int64_t e = b0; e < b1; ++e)
                    if (e == b0 || !ent[e].same_edge(ent[e - 1])) ++r;
                brows[m + 1] = r;
            }
        }
    });
    tr.mark("closedness sort");
    for (int m = 0; m < nvx; ++m) brows[m + 1] += brows[m];
    const int64_t n_closed = brows[nvx];
    P->n_closed = n_closed;
    // room for the projection rows and the end mark, so that appending them moves nothing
    P->row_ptr.reserve(size_t(n_closed) + size_t(X.nt) + size_t(Y.nt) + 1);
    P->row_ptr.resize(size_t(n_closed));  // every row start is written below
    // projection entries: elements whose X (Y) side is a triangle; all rows are sized once
    std::vector<int64_t> nproj_part(size_t(nth), 0);
    parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
        int64_t k = 0;
        for (int64_t i = lo; i < hi; ++i) k += (E.type[i] == 0) ? 2 : 1;
        nproj_part[size_t(c)] += k;
    });
    int64_t nproj_entries = 0;
    for (int64_t k : nproj_part) nproj_entries += k;
    P->row_var.resize(size_t(ne + nproj_entries));
    P->row_coef.resize(size_t(ne + nproj_entries));
    pod_vector<int32_t> row_ent(static_cast<size_t>(ne + nproj_entries));  // corner (0..2) or 3 + side
    // the rows of every element in one record (presolve reads all of them per fixing):
    // closed[v] = closedness row of corner v << 1 | (coefficient there > 0), filled after the
    // dense presolve rounds for the variables still free; proj[side] = the X / Y projection
    // row, -1 if none
    struct ElemRows {
        uint32_t closed[3];
        int32_t proj[2];
    };
    pod_vector<ElemRows> er(static_cast<size_t>(nv));
    // presolve state of every row: residual right-hand side, free +1 / -1 entries
    struct RowState {
        int32_t res, np, nn, queued;
    };
    pod_vector<RowState> rs(static_cast<size_t>(n_closed + X.nt + Y.nt));
    // right-hand sides: 0 for the closedness rows (written by the fill below, in parallel),
    // 1 for the projection rows appended later
    P->rhs.reserve(size_t(n_closed) + size_t(X.nt) + size_t(Y.nt));
    P->rhs.resize(size_t(n_closed));
    tr.mark("closedness arrays");
    parallel_chunks(nvx, nth * 4, [&](int, int64_t lo, int64_t hi) {
        for (int64_t m = lo; m < hi; ++m) {
            int64_t r = brows[m] - 1;
            for (int64_t e = bstart[m]; e < bstart[m + 1]; ++e) {
                if (e == bstart[m] || !ent[e].same_edge(ent[e - 1])) {
                    P->row_ptr[++r] = e;
                    rs[r] = RowState{0, 0, 0, 0};
                    P->rhs[size_t(r)] = 0;
                }
                const uint32_t id = ent[e].id >> 1;
                const bool neg = ent[e].id & 1u;
                P->row_var[e] = int32_t(id / 3);
                P->row_coef[e] = neg ? -1 : 1;
                row_ent[e] = int32_t(id % 3);
                ++(neg ? rs[r].nn : rs[r].np);
            }
        }
    });
    pod_vector<EdgeEntry>().swap(ent);

    tr.mark("closedness rows");
    // ---- projection rows (counting sort keeps the element order inside a row): one row per X
    // triangle, then one per Y triangle; one counting and one scatter pass serve both sides
    const int ntx = X.nt, ntri = X.nt + Y.nt;        // row t: X triangle t, or Y triangle t - ntx
    auto tris_of = [&](int64_t i, int* a, int* b) {
        const int ty = E.type[i];
        *a = (ty == 0 || ty == 1 || ty == 3) ? E.xe[i] : -1;
        *b = (ty == 0 || ty == 2 || ty == 4) ? ntx + E.ye[i] : -1;
    };
    std::vector<std::vector<int64_t>> pcnt(nth, std::vector<int64_t>(size_t(ntri), 0));
    parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
        int64_t* k = pcnt[c].data();
        for (int64_t i = lo; i < hi; ++i) {
            int a, b;
            tris_of(i, &a, &b);
            if (a >= 0) ++k[a];
            if (b >= 0) ++k[b];
        }
    });
    const int64_t row0 = int64_t(P->row_ptr.size());
    std::vector<std::vector<int64_t>> poff(nth, std::vector<int64_t>(size_t(ntri), 0));
    int64_t proj_end = ne;
    for (int t = 0; t < ntri; ++t) {
        int64_t tot = 0;
        for (int c = 0; c < nth; ++c) tot += pcnt[c][t];
        if (tot == 0) { *err = "a triangle has no matching element"; return DISCO_ERR_INFEASIBLE; }
        rs[size_t(row0 + t)] = RowState{1, int32_t(tot), 0, 0};
        P->row_ptr.push_back(proj_end);
        for (int c = 0; c < nth; ++c) {
            poff[c][t] = proj_end;
            proj_end += pcnt[c][t];
        }
    }
    parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
        int64_t* o = poff[c].data();
        for (int64_t i = lo; i < hi; ++i) {
            int ab[2];
            tris_of(i, &ab[0], &ab[1]);
            for (int side = 0; side < 2; ++side) {
                const int t = ab[side];
                er[size_t(i)].proj[side] = t >= 0 ? int32_t(row0 + t) : -1;
                if (t >= 0) P->row_var[size_t(o[t]++)] = int32_t(i);
            }
        }
    });
    // coefficients (all +1) and entry codes (3 + side) of the projection entries, in order
    {
        const int64_t ybeg = P->row_ptr[size_t(row0 + ntx)];
        parallel_chunks(proj_end - ne, nth, [&](int, int64_t lo, int64_t hi) {
            for (int64_t k = ne + lo; k < ne + hi; ++k) {
                P->row_coef[size_t(k)] = 1;
                row_ent[size_t(k)] = k < ybeg ? 3 : 4;
            }
        });
    }
    P->rhs.resize(P->rhs.size() + size_t(ntri), 1);
    P->n_projx = X.nt;
    P->n_projy = Y.nt;
    P->nrows = int64_t(P->rhs.size());
    P->row_region.resize(size_t(P->nrows));
    parallel_chunks(nvx, nth, [&](int, int64_t m0, int64_t m1) {
        for (int64_t m = m0; m < m1; ++m)
            std::fill(P->row_region.begin() + brows[m], P->row_region.begin() + brows[m + 1], int32_t(m));
    });
    for (int t = 0; t < X.nt; ++t)
        P->row_region[size_t(n_closed + t)] = std::min({X.T[3 * t], X.T[3 * t + 1], X.T[3 * t + 2]});
    for (int t = 0; t < Y.nt; ++t) P->row_region[size_t(n_closed + X.nt + t)] = nvx + t;
    if (proj_end != int64_t(P->row_var.size())) { *err = "internal: projection entry count"; return DISCO_ERR_INVALID_ARG; }
    P->row_ptr.push_back(proj_end);
    const int64_t nr = P->nrows;

    tr.mark("projection rows");
    // row chunks of about equal entry counts (projection rows are long, closedness rows
    // short), taken dynamically by the threads; the results do not depend on the chunking
    const int64_t n_entries = P->row_ptr[size_t(nr)];
    const int nrc = std::max(1, std::min<int>(nth * 8, int(nr / 1024) + 1));
    std::vector<int64_t> row_cut(size_t(nrc) + 1, nr);
    row_cut[0] = 0;
    for (int c = 1; c < nrc; ++c) {
        const int64_t want = n_entries * c / nrc;
        row_cut[size_t(c)] = std::max<int64_t>(
            row_cut[size_t(c) - 1],
            int64_t(std::lower_bound(P->row_ptr.begin(), P->row_ptr.begin() + nr, want) - P->row_ptr.begin()));
    }
    // ---- presolve: saturated rows force all their free variables, to a fixpoint. Rows and
    // variables are split into contiguous ranges, one per thread, and each thread alone
    // writes the state of its ranges. A round is bulk-synchronous: (1) the owners of the
    // frontier rows decide on the counts of the previous round and send every forced value
    // to the variable's owner; (2) variable owners fix the variables (a second, different
    // value is a conflict) and send (row, coefficient, value) to the owners of the
    // variable's rows; (3) row owners update the free counts and the residual and queue each
    // updated row once for the next round. The fixed values are the unique arc-consistent
    // closure whatever the thread count and whatever the order of the rounds.
    //
    // While a round fixes many variables (the first rounds fix most of the ones presolve
    // fixes), dense rounds do the same work with sequential access: every acting row flags
    // the values it forces (one flag per value, so a variable flagged both ways is a
    // conflict; plain stores, no read-modify-write), the flags become fixings, and every row's
    // residual and free counts are recounted from its entries. The incremental rounds then
    // continue from the recounted state.
    P->fixed.assign(size_t(nv), -1);
    int dense_rounds = 0;
    bool dense_conflict = false;
    {
        std::vector<uint8_t> to0(static_cast<size_t>(nv), 0), to1(static_cast<size_t>(nv), 0);
        std::atomic<bool> bad{false};
        std::vector<int64_t> nfix(static_cast<size_t>(nth), 0);
        for (;;) {
            // (1) decide: a first round acts on every saturated or violated row (nothing is
            // fixed yet), later ones on those with free entries
            const bool first = dense_rounds == 0;
            parallel_tasks(nrc, nth, [&](int64_t c) {
                for (int64_t r = row_cut[size_t(c)]; r < row_cut[size_t(c) + 1]; ++r) {
                    const RowState q = rs[r];
                    if (q.np + q.nn == 0) {
                        if (first && q.res != 0) bad.store(true, std::memory_order_relaxed);
                        continue;
                    }
                    if (q.res > q.np || q.res < -q.nn) {
                        bad.store(true, std::memory_order_relaxed);
                        continue;
                    }
                    int up;
                    if (q.res == q.np) up = 1;
                    else if (q.res == -q.nn) up = 0;
                    else continue;
                    for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
                        const int32_t v = P->row_var[e];
                        if (P->fixed[v] >= 0) continue;
                        const bool one = (P->row_coef[e] > 0) == (up == 1);
                        __atomic_store_n(one ? &to1[size_t(v)] : &to0[size_t(v)], uint8_t(1), __ATOMIC_RELAXED);
                    }
                }
            });
            ++dense_rounds;
            if (bad.load()) {
                dense_conflict = true;
                break;
            }
            // (2) the flags become fixings
            std::vector<uint8_t> clash(static_cast<size_t>(nth), 0);
            parallel_chunks(nv, nth, [&](int c, int64_t lo, int64_t hi) {
                int64_t k = 0;
                uint8_t x = 0;
                for (int64_t v = lo; v < hi; ++v) {
                    const uint8_t a = to0[size_t(v)], b = to1[size_t(v)];
                    x |= a & b;
                    P->fixed[size_t(v)] = b ? int8_t(1) : (a ? int8_t(0) : P->fixed[size_t(v)]);
                    to0[size_t(v)] = 0;
                    to1[size_t(v)] = 0;
                    k += a | b;
                }
                nfix[size_t(c)] = k;
                clash[size_t(c)] = x;
            });
            if (std::find(clash.begin(), clash.end(), uint8_t(1)) != clash.end()) {
                dense_conflict = true;
                break;
            }
            int64_t fixed_now = 0;
            for (int64_t k : nfix) fixed_now += k;
            if (tr.on) std::fprintf(stderr, "disco build  dense round %d fixes %lld\n", dense_rounds, (long long)fixed_now);
            if (fixed_now == 0) break;  // no row acts: the state is already the closure's
            // (3) recount every row that had free entries from its entries
            parallel_tasks(nrc, nth, [&](int64_t c) {
                for (int64_t r = row_cut[size_t(c)]; r < row_cut[size_t(c) + 1]; ++r) {
                    if (rs[r].np + rs[r].nn == 0) continue;
                    int32_t res = P->rhs[size_t(r)], np = 0, nf = 0;  // branch-free: fixings look random
                    for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
                        const int32_t f = P->fixed[P->row_var[e]];
                        const int32_t c = P->row_coef[e];
                        nf += f < 0;
                        np += (f < 0) & (c > 0);
                        res -= c * (f == 1);
                    }
                    rs[r] = RowState{res, np, nf - np, 0};
                }
            });
            // each fixing updates about five rows in an incremental round
            if (5 * fixed_now < n_entries / 8) break;
        }
    }
    tr.mark("presolve dense");
    if (!dense_conflict) {
        // closedness rows of the variables still free (only the incremental rounds use them)
        parallel_tasks(nrc, nth, [&](int64_t c) {
            for (int64_t r = row_cut[size_t(c)]; r < std::min(row_cut[size_t(c) + 1], n_closed); ++r)
                for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1] && rs[r].np + rs[r].nn > 0; ++e) {
                    const int32_t v = P->row_var[e];
                    if (P->fixed[v] < 0)
                        er[size_t(v)].closed[row_ent[e]] = uint32_t(r) << 1 | (P->row_coef[e] > 0 ? 1u : 0u);
                }
        });
        tr.mark("free closedness rows");
    }
    if (!dense_conflict) {
        const int nt = nth;
        // owner of row r / variable v: table lookup by blocks of 4096
        auto owners = [&](int64_t n) {
            std::vector<uint8_t> tab(size_t((n >> 12) + 1));
            for (size_t b = 0; b < tab.size(); ++b) tab[b] = uint8_t(std::min<int64_t>(nt - 1, (int64_t(b) << 12) * nt / n));
            return tab;
        };
        if (nt > 255) { *err = "too many host threads"; return DISCO_ERR_INVALID_ARG; }
        const std::vector<uint8_t> row_owner = owners(nr), var_owner = owners(nv);
        auto row_lo = [&](int t) {  // first row owned by t (block granular, matches the table)
            int64_t b = 0;
            while (b < int64_t(row_owner.size()) && row_owner[b] < t) ++b;
            return std::min<int64_t>(nr, b << 12);
        };
        std::vector<std::vector<int32_t>> frontier(nt);
        parallel_chunks(nt, nt, [&](int t, int64_t, int64_t) {
            // rows with free entries that are saturated or violated after the dense rounds
            for (int64_t r = row_lo(t), r1 = row_lo(t + 1); r < r1; ++r)
                if (rs[r].np + rs[r].nn > 0 && (rs[r].res >= rs[r].np || rs[r].res <= -rs[r].nn))
                    frontier[t].push_back(int32_t(r));
        });
        struct Upd {
            int32_t row;
            int32_t code;  // bit 0: value, bit 1: coefficient > 0
        };
        std::vector<std::vector<std::vector<std::pair<int32_t, int8_t>>>> force(nt, std::vector<std::vector<std::pair<int32_t, int8_t>>>(nt));
        std::vector<std::vector<std::vector<Upd>>> upd(nt, std::vector<std::vector<Upd>>(nt));
        std::vector<int> bad(nt, 0);
        auto any = [&](auto pred) {
            for (int t = 0; t < nt; ++t)
                if (pred(t)) return true;
            return false;
        };
        tr.mark("presolve setup");
        int rounds = 0;
        while (any([&](int t) { return !frontier[t].empty(); })) {
            if (tr.on && rounds < 4) {
                char what[32];
                std::snprintf(what, sizeof(what), "presolve round %d", rounds);
                tr.mark(what);
            }
            ++rounds;
            // (1) decide
            parallel_chunks(nt, nt, [&](int t, int64_t, int64_t) {
                for (auto& b : force[t]) b.clear();
                for (const int32_t r : frontier[t]) {
                    RowState& q = rs[r];
                    q.queued = 0;
                    if (q.res > q.np || q.res < -q.nn) { bad[t] = 1; return; }
                    if (q.np + q.nn == 0) continue;
                    int up;
                    if (q.res == q.np) up = 1;
                    else if (q.res == -q.nn) up = 0;
                    else continue;
                    for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
                        const int32_t v = P->row_var[e];
                        if (P->fixed[v] < 0)
                            force[t][var_owner[size_t(v) >> 12]].emplace_back(v, int8_t(P->row_coef[e] > 0 ? up : 1 - up));
                    }
                }
            });
            if (any([&](int t) { return bad[t] != 0; })) break;
            // (2) fix
            parallel_chunks(nt, nt, [&](int u, int64_t, int64_t) {
                for (auto& b : upd[u]) b.clear();
                for (int t = 0; t < nt; ++t)
                    for (auto [v, val] : force[t][u]) {
                        const int8_t f = P->fixed[v];
                        if (f == val) continue;
                        if (f >= 0) { bad[u] = 1; return; }
                        P->fixed[v] = val;
                        const ElemRows& x = er[size_t(v)];
                        for (int q = 0; q < 3; ++q) {
                            const int32_t r = int32_t(x.closed[q] >> 1);
                            upd[u][row_owner[size_t(r) >> 12]].push_back(Upd{r, val | ((x.closed[q] & 1u) ? 2 : 0)});
                        }
                        for (int side = 0; side < 2; ++side) {
                            const int32_t r = x.proj[side];
                            if (r >= 0) upd[u][row_owner[size_t(r) >> 12]].push_back(Upd{r, val | 2});
                        }
                    }
            });
            if (any([&](int t) { return bad[t] != 0; })) break;
            // (3) update the rows, queue each once
            parallel_chunks(nt, nt, [&](int t, int64_t, int64_t) {
                frontier[t].clear();
                for (int u = 0; u < nt; ++u)
                    for (const Upd& m : upd[u][t]) {
                        RowState& q = rs[m.row];
                        if (m.code & 2) {
                            --q.np;
                            q.res -= m.code & 1;
                        } else {
                            --q.nn;
                            q.res += m.code & 1;
                        }
                        // only a saturated (or violated) row with free entries can act; a
                        // saturated row stays saturated or turns violated under further
                        // fixings, so testing after each update misses none. Rows left without
                        // free entries are checked once after the fixpoint.
                        if (!q.queued && q.np + q.nn > 0 && (q.res >= q.np || q.res <= -q.nn)) {
                            q.queued = 1;
                            frontier[t].push_back(m.row);
                        }
                    }
            });
        }
        if (any([&](int t) { return bad[t] != 0; })) { *err = "presolve: a row has no solution"; return DISCO_ERR_INFEASIBLE; }
        if (tr.on) std::fprintf(stderr, "disco build  presolve rounds: %d dense + %d\n", dense_rounds, rounds);
    }
    if (dense_conflict) { *err = "presolve: a row has no solution"; return DISCO_ERR_INFEASIBLE; }
    {
        std::atomic<bool> violated{false};
        parallel_chunks(nr, nth, [&](int, int64_t lo, int64_t hi) {
            for (int64_t r = lo; r < hi; ++r)
                if (rs[r].np + rs[r].nn == 0 && rs[r].res != 0) violated.store(true, std::memory_order_relaxed);
        });
        if (violated.load()) { *err = "presolve: violated row"; return DISCO_ERR_INFEASIBLE; }
    }
    tr.mark("presolve");
    // internal ids of the free variables in element order, and the constant (costs of the
    // variables fixed to 1), over fixed-size blocks so that the sums do not depend on the
    // thread count
    pod_vector<int32_t> internal(static_cast<size_t>(nv));
    {
        constexpr int64_t kBlock = int64_t(1) << 16;
        const int64_t nb = (nv + kBlock - 1) / kBlock;
        std::vector<int64_t> nfree(size_t(nb) + 1, 0);
        std::vector<double> part(size_t(nb), 0.0);
        parallel_chunks(nb, nth, [&](int, int64_t b0, int64_t b1) {
            for (int64_t b = b0; b < b1; ++b) {
                int64_t k = 0;
                double c = 0.0;
                for (int64_t i = b * kBlock; i < std::min(nv, (b + 1) * kBlock); ++i) {
                    if (P->fixed[i] == 1) c += P->cost[i];
                    k += P->fixed[i] < 0;
                }
                nfree[size_t(b) + 1] = k;
                part[size_t(b)] = c;
            }
        });
        P->constant = 0.0;
        for (int64_t b = 0; b < nb; ++b) {
            nfree[size_t(b) + 1] += nfree[size_t(b)];
            P->constant += part[size_t(b)];
        }
        P->free_orig.resize(size_t(nfree[size_t(nb)]));
        parallel_chunks(nb, nth, [&](int, int64_t b0, int64_t b1) {
            for (int64_t b = b0; b < b1; ++b) {
                int64_t k = nfree[size_t(b)];
                for (int64_t i = b * kBlock; i < std::min(nv, (b + 1) * kBlock); ++i) {
                    if (P->fixed[i] < 0) {
                        internal[size_t(i)] = int32_t(k);
                        P->free_orig[size_t(k++)] = int32_t(i);
                    } else {
                        internal[size_t(i)] = -1;
                    }
                }
            }
        });
    }
    P->n_free = int64_t(P->free_orig.size());

    tr.mark("internal ids");
    // ---- BDD segments, compiled in parallel over row ranges; slot rank = which of the
    // variable's rows this is (closedness corner 0..2, then projection rows), so it is known
    // locally; auxiliaries get rank 0 in the left segment and 1 in the right one
    // degree: every free element keeps all its rows (3 closedness + its projection rows); an
    // auxiliary variable sits in two segments
    std::vector<uint8_t> deg_free(static_cast<size_t>(P->n_free));
    parallel_chunks(P->n_free, nth, [&](int, int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; ++v) {
            const int64_t i = P->free_orig[v];
            deg_free[v] = uint8_t(3 + (er[size_t(i)].proj[0] >= 0) + (er[size_t(i)].proj[1] >= 0));
        }
    });
    std::vector<RowChunk> chunks(nrc);
    parallel_tasks(nrc, nth, [&](int64_t c) {
        std::vector<int32_t> fv, lo, wd;
        std::vector<int8_t> fc;
        std::vector<uint8_t> fr;
        std::vector<int64_t> cut_aux;  // local id of y_1 of the cut before segment s
        {
            RowChunk& C = chunks[c];
            const int64_t r0 = row_cut[size_t(c)], r1 = row_cut[size_t(c) + 1];
            // about one slot per entry (fixed entries drop out, split chains add a few)
            C.var.reserve(size_t(P->row_ptr[size_t(r1)] - P->row_ptr[size_t(r0)]));
            C.desc.reserve(C.var.capacity());
            auto add_slot = [&](int32_t var, int w, int wn, int d0, int d1, bool one, int rank) {
                C.var.push_back(var);
                C.desc.push_back(pack_desc(w, wn, d0, d1, one, rank, var < 0 ? 2 : deg_free[var]));
                C.nodes += w;
            };
            for (int64_t r = r0; r < r1 && !C.rc; ++r) {
                if (rs[r].np + rs[r].nn == 0) continue;  // presolve left no free entry (its counts are exact)
                fv.clear();
                fc.clear();
                fr.clear();
                for (int64_t e = P->row_ptr[r]; e < P->row_ptr[r + 1]; ++e) {
                    const int32_t v = P->row_var[e];
                    if (P->fixed[v] >= 0) continue;
                    fv.push_back(internal[v]);
                    fc.push_back(P->row_coef[e]);
                    // projection rank: 3 for the first projection row of the element, 4 for the second
                    int rk = row_ent[e];
                    if (rk == 4 && er[size_t(v)].proj[0] < 0) rk = 3;
                    fr.push_back(uint8_t(rk));
                }
                const int n = int(fv.size());
                if (n == 0) continue;
                const int rr = rs[r].res;
                int ptot = 0, qtot = 0;
                for (int8_t cf : fc) (cf > 0 ? ptot : qtot)++;
                lo.assign(n + 1, 0);
                wd.assign(n + 1, 0);
                int ppre = 0, qpre = 0;
                for (int l = 0; l <= n; ++l) {
                    lo[l] = std::max(-qpre, rr - (ptot - ppre));
                    wd[l] = std::min(ppre, rr + (qtot - qpre)) - lo[l] + 1;
                    if (wd[l] < 1 || wd[l] > kMaxWidth) {
                        C.err = wd[l] < 1 ? "empty BDD layer after presolve" : "BDD layer wider than 32 nodes";
                        C.rc = wd[l] < 1 ? DISCO_ERR_INFEASIBLE : DISCO_ERR_INVALID_ARG;
                        break;
                    }
                    if (l < n) (fc[l] > 0 ? ppre : qpre)++;
                }
                if (C.rc) break;
                int nseg = (split_chunk > 0 && n > split_chunk) ? (n + split_chunk - 1) / split_chunk : 1;
                if (split_max_segments > 0) nseg = std::min(nseg, split_max_segments);
                cut_aux.assign(size_t(nseg) + 1, -1);
                for (int s = 1; s < nseg; ++s) {
                    const int b = int(int64_t(s) * n / nseg);
                    if (wd[b] > 1) {
                        if (wd[b] + 1 > kMaxWidth) { C.err = "split layer too wide"; C.rc = DISCO_ERR_INVALID_ARG; break; }
                        cut_aux[s] = C.n_aux;
                        C.n_aux += wd[b];
                    }
                }
                if (C.rc) break;
                for (int s = 0; s < nseg; ++s) {
                    const int b0 = int(int64_t(s) * n / nseg), b1 = int(int64_t(s + 1) * n / nseg);
                    Segment sg{r, s, int64_t(C.var.size()), 0, 0};
                    if (s > 0 && wd[b0] > 1) {  // prefix chain: read the one-hot y_1..y_k, enter node j
                        const int k = wd[b0];
                        for (int j = 1; j <= k; ++j) {
                            const int32_t var = int32_t(-1 - (cut_aux[s] + j - 1));
                            if (j < k) add_slot(var, j, j + 1, 0, j, true, 1);
                            else add_slot(var, k, k, -1, k - 1, true, 1);
                            sg.max_width = std::max(sg.max_width, j);
                        }
                    }
                    for (int l = b0; l < b1; ++l) {
                        const int d0 = lo[l] - lo[l + 1];
                        add_slot(fv[l], wd[l], wd[l + 1], d0, d0 + fc[l], false, fr[l]);
                        sg.max_width = std::max(sg.max_width, wd[l]);
                    }
                    if (s + 1 < nseg && wd[b1] > 1) {  // suffix chain: y_j = 1 iff the path leaves through node j
                        const int k = wd[b1];
                        for (int j = 1; j <= k; ++j) {
                            const int32_t var = int32_t(-1 - (cut_aux[s + 1] + j - 1));
                            const int w = j == 1 ? k : k - j + 2;
                            add_slot(var, w, j < k ? k - j + 1 : 1, -1, k - j, true, 0);
                            sg.max_width = std::max(sg.max_width, w);
                        }
                    }
                    sg.n_layers = int32_t(int64_t(C.var.size()) - sg.first_slot);
                    C.max_layers = std::max(C.max_layers, sg.n_layers);
                    C.max_width = std::max(C.max_width, sg.max_width);
                    C.segs.push_back(sg);
                }
            }
        }
    });
    for (const RowChunk& C : chunks)
        if (C.rc) { *err = C.err; return C.rc; }
    tr.mark("bdd segments");
    // global offsets of slots, segments and auxiliaries per chunk
    std::vector<int64_t> slot_off(nrc + 1, 0), seg_off(nrc + 1, 0), aux_off(nrc + 1, 0);
    int64_t nodes = 0;
    int max_layers = 0, max_width = 0;
    for (int c = 0; c < nrc; ++c) {
        slot_off[c + 1] = slot_off[c] + int64_t(chunks[c].var.size());
        seg_off[c + 1] = seg_off[c] + int64_t(chunks[c].segs.size());
        aux_off[c + 1] = aux_off[c] + chunks[c].n_aux;
        nodes += chunks[c].nodes;
        max_layers = std::max(max_layers, chunks[c].max_layers);
        max_width = std::max(max_width, chunks[c].max_width);
    }
    P->n_aux = aux_off[nrc];
    const int64_t nint = P->n_free + P->n_aux;
    if (nint >= (int64_t(1) << 31)) { *err = "too many variables"; return DISCO_ERR_INVALID_ARG; }
    const int64_t ns = slot_off[nrc];
    P->slot_var.resize(size_t(ns));
    P->slot_desc.resize(size_t(ns));
    P->slot_lam0.resize(size_t(ns));
    P->slot_lam0_lo.resize(size_t(ns));
    P->segs.resize(size_t(seg_off[nrc]));
    P->deg.assign(size_t(nint), 2);
    std::copy(deg_free.begin(), deg_free.end(), P->deg.begin());
    parallel_tasks(nrc, nth, [&](int64_t c) {
        {
            const RowChunk& C = chunks[c];
            const int64_t so = slot_off[c];
            for (size_t i = 0; i < C.var.size(); ++i) {
                int32_t v = C.var[i];
                if (v < 0) v = int32_t(P->n_free + aux_off[c] + (-1 - int64_t(v)));
                const int dg = P->deg[v];
                P->slot_var[so + i] = v;
                P->slot_desc[so + i] = C.desc[i];
                const double l0 = v < P->n_free ? P->cost[P->free_orig[v]] / dg : 0.0;
                P->slot_lam0[so + i] = float(l0);
                P->slot_lam0_lo[so + i] = float(l0 - double(float(l0)));
            }
            for (size_t k = 0; k < C.segs.size(); ++k) {
                Segment sg = C.segs[k];
                sg.first_slot += so;
                P->segs[seg_off[c] + k] = sg;
            }
        }
    });
    tr.mark("slot arrays");
    P->n_nodes = nodes;
    P->max_layers = max_layers;
    P->max_width = max_width;
    P->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return DISCO_OK;
}

}  // namespace disco
