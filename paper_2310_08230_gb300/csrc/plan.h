// Host-side compilation of ILP (P) into BDD segments ("the plan"), consumed by the device
// store in disco.cu. See host_build.cpp for the passages each step follows.
#pragma once

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

namespace disco {

// Large host blocks (pod_vector storage: the compiled plans and the compiler's work
// arrays) come from a process-wide cache. A build that follows a freed one of similar size
// reuses its pages instead of faulting in, and having the kernel zero, hundreds of MB of
// fresh memory, and a free returns the pages to the cache instead of unmapping them.
// Blocks of at least 1 MB are rounded up to a size class (an eighth of a power of two) and
// kept up to a total of DISCO_HOST_CACHE_MB megabytes (default 2048; 0 turns the cache off).
void* host_block_alloc(size_t bytes);
void host_block_free(void* p, size_t bytes) noexcept;

// Allocator that leaves trivially constructible elements uninitialised on resize, so that large
// arrays are first touched by the (parallel) code that fills them instead of being zeroed.
template <class T>
struct uninit_alloc : std::allocator<T> {
    using value_type = T;
    template <class U>
    struct rebind {
        using other = uninit_alloc<U>;
    };
    uninit_alloc() = default;
    template <class U>
    uninit_alloc(const uninit_alloc<U>&) noexcept {}
    T* allocate(size_t n) {
        if (n > size_t(-1) / sizeof(T)) throw std::bad_array_new_length();
        return static_cast<T*>(host_block_alloc(n * sizeof(T)));
    }
    void deallocate(T* p, size_t n) noexcept { host_block_free(p, n * sizeof(T)); }
    template <class U>
    void construct(U* p) noexcept {
        ::new (static_cast<void*>(p)) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
    }
};
template <class T>
using pod_vector = std::vector<T, uninit_alloc<T>>;

// Persistent worker threads for parallel_chunks (creating and joining threads for every
// parallel phase costs tens of microseconds per thread on many-core hosts). One job at a
// time; its tasks are taken dynamically by the workers and the calling thread. A worker
// checks into a job under the lock and out when it finds no task left; the caller returns
// only when every task has finished and every worker that checked in has checked out, so no
// worker ever touches a finished job.
class WorkerPool {
public:
    static WorkerPool& get() {
        static WorkerPool pool(int(std::max(2u, std::thread::hardware_concurrency())) - 1);
        return pool;
    }
    // Runs f(0 .. n-1); false (nothing run) if the pool is busy or called from a worker.
    bool try_run(int n, const std::function<void(int)>& f) {
        if (in_worker() || !busy_.try_lock()) return false;
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            njobs_ = n;
            next_.store(0);
            remaining_ = n;
            ++gen_;
        }
        cv_.notify_all();
        run_tasks(f, n);
        {
            std::unique_lock<std::mutex> lk(mu_);
            done_.wait(lk, [&] { return remaining_ == 0 && active_ == 0; });
            job_ = nullptr;
        }
        busy_.unlock();
        return true;
    }
    ~WorkerPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : threads_) t.join();
    }

private:
    explicit WorkerPool(int nthreads) {
        for (int i = 0; i < nthreads; ++i)
            threads_.emplace_back([this] {
                in_worker() = true;
                uint64_t seen = 0;
                for (;;) {
                    const std::function<void(int)>* f = nullptr;
                    int n = 0;
                    {
                        std::unique_lock<std::mutex> lk(mu_);
                        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                        if (stop_) return;
                        seen = gen_;
                        if (!job_) continue;
                        f = job_;
                        n = njobs_;
                        ++active_;  // check in
                    }
                    run_tasks(*f, n);
                    std::lock_guard<std::mutex> lk(mu_);
                    if (--active_ == 0 && remaining_ == 0) done_.notify_all();  // check out
                }
            });
    }
    static bool& in_worker() {
        static thread_local bool flag = false;
        return flag;
    }
    void run_tasks(const std::function<void(int)>& f, int n) {
        for (int i; (i = next_.fetch_add(1)) < n;) {
            f(i);
            std::lock_guard<std::mutex> lk(mu_);
            if (--remaining_ == 0 && active_ == 0) done_.notify_all();
        }
    }
    std::vector<std::thread> threads_;
    std::mutex mu_, busy_;
    std::condition_variable cv_, done_;
    const std::function<void(int)>* job_ = nullptr;
    int njobs_ = 0, remaining_ = 0, active_ = 0;
    std::atomic<int> next_{0};
    uint64_t gen_ = 0;
    bool stop_ = false;
};

// Runs body(chunk, lo, hi) over [0, n) split into `nch` contiguous chunks in parallel.
template <class F>
inline void parallel_chunks(int64_t n, int nch, F body) {
    if (nch <= 1 || n < 2) {
        body(0, int64_t(0), n);
        return;
    }
    const std::function<void(int)> task = [&](int c) { body(c, n * c / nch, n * (c + 1) / nch); };
    if (WorkerPool::get().try_run(nch, task)) return;
    std::vector<std::thread> pool;
    for (int c = 0; c < nch; ++c) pool.emplace_back([&task, c] { task(c); });
    for (auto& th : pool) th.join();
}

// Runs body(i) for i in [0, n) as dynamically scheduled tasks on up to nth threads (in
// order on the calling thread when nth <= 1 or called from inside a pool task).
template <class F>
inline void parallel_tasks(int64_t n, int nth, F body) {
    if (nth <= 1 || n < 2) {
        for (int64_t i = 0; i < n; ++i) body(i);
        return;
    }
    const std::function<void(int)> task = [&](int i) { body(int64_t(i)); };
    if (WorkerPool::get().try_run(int(n), task)) return;
    std::atomic<int64_t> next{0};
    auto worker = [&] {
        for (int64_t i; (i = next.fetch_add(1)) < n;) body(i);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < std::min<int64_t>(nth, n); ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

// Phase timer: with DISCO_TRACE set in the environment, each phase's wall time goes to stderr.
struct Trace {
    const char* scope = "build";
    bool on = std::getenv("DISCO_TRACE") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void mark(const char* phase) {
        if (!on) return;
        const auto n = std::chrono::steady_clock::now();
        std::fprintf(stderr, "disco %-6s %-22s %8.2f ms\n", scope, phase,
                     std::chrono::duration<double, std::milli>(n - t).count());
        t = n;
    }
};

// Widest BDD layer the device kernels accept (node states held in registers).
constexpr int kMaxWidth = 32;

// Per-slot layer descriptor (uint32):
//   bits  0..5   w     nodes in this layer (1..32)
//   bits  6..11  wn    nodes in the next layer (1..32); the terminal layer has 1 node
//   bits 12..14  d0+2  0-arc: node s goes to node s + d0 of the next layer
//   bits 15..20  d1+2  1-arc: node s goes to node s + d1 (d1 in [-2, 32])
//   bit  21      one   the 1-arc leaves only node 0 (auxiliary chains of a split)
//   bits 22..24  rank  position of this slot among its variable's slots
//   bits 25..27  deg   number of slots of the variable (|J_i|, 2..5)
// An arc whose target index falls outside [0, wn) leads to the false terminal.
inline uint32_t pack_desc(int w, int wn, int d0, int d1, bool one, int rank, int deg) {
    return uint32_t(w - 1) | (uint32_t(wn - 1) << 6) | (uint32_t(d0 + 2) << 12) |
           (uint32_t(d1 + 2) << 15) | (uint32_t(one ? 1 : 0) << 21) | (uint32_t(rank) << 22) |
           (uint32_t(deg) << 25);
}

struct Segment {
    int64_t row;        // row of (P)
    int32_t index;      // segment index within the row
    int64_t first_slot; // canonical index of its first layer
    int32_t n_layers;
    int32_t max_width;
};

struct Plan {
    // ---- problem (P)
    int32_t nvx = 0, nvy = 0;
    int64_t nvars = 0, nrows = 0, n_closed = 0, n_projx = 0, n_projy = 0;
    pod_vector<int32_t> vm, vn;         // 3 per variable: X / Y vertex of each corner
    pod_vector<double> cost;            // c_p per variable (normalised unless disabled)
    double cost_scale = 1.0;            // c_p = (mean of its pair costs) / cost_scale
    double cost_max = 0.0;              // largest c_p (1 when normalised)
    int64_t cost_scale_elem = -1;       // the element whose raw cost is cost_scale (normalised)
    std::vector<double> area_x, area_y; // cost model 1 (Eq. 2): mixed vertex areas; else empty
    // per row, the mesh region its variables sit in (a tile-order key): a closedness row the
    // X vertex of its bucket, an X projection row its triangle's smallest X vertex, a Y
    // projection row nvx + its Y triangle (Y rows gather elements from all over X)
    pod_vector<int32_t> row_region;
    pod_vector<int64_t> row_ptr;        // rows: closedness, X projection, Y projection
    pod_vector<int32_t> row_var;
    pod_vector<int8_t> row_coef;
    pod_vector<int32_t> rhs;
    // ---- presolve
    std::vector<int8_t> fixed;           // per variable: -1 free, 0 / 1 fixed
    double constant = 0.0;               // sum of c over variables fixed to 1
    // ---- internal variables: [0, n_free) free variables in ascending id, then auxiliaries
    int64_t n_free = 0, n_aux = 0;
    std::vector<int32_t> free_orig;      // internal id -> variable id (free ones)
    std::vector<uint8_t> deg;            // slots per internal variable
    // ---- canonical slots: segments by (row, index), layers in order
    pod_vector<int32_t> slot_var;       // internal variable id
    pod_vector<uint32_t> slot_desc;
    pod_vector<float> slot_lam0;        // lambda^0 = c / |J| (high part), 0 for auxiliaries
    pod_vector<float> slot_lam0_lo;     // low part: c / |J| - slot_lam0
    std::vector<Segment> segs;
    int64_t n_nodes = 0;
    int32_t max_layers = 0, max_width = 0;
    double build_ms = 0.0;
};

struct MeshIn {
    int32_t nv, nt;
    const int32_t* T;
    const float* V = nullptr;  // nv x 3 positions (needed by cost model 1 only)
};

// Mixed (Voronoi) area of every vertex of a triangle mesh (Eq. 2's A, after Meyer et al.
// 2003): per triangle, a non-obtuse triangle gives each corner its Voronoi part
// (|PR|^2 cot Q + |PQ|^2 cot R) / 8; an obtuse one gives half its area to the obtuse corner
// and a quarter to each other corner.
void mixed_areas(const MeshIn& M, std::vector<double>* out);

// Returns 0 or a negative DISCO_ERR_* code (err receives a message).
// cost_model 0: c_p = mean of the element's three pair costs; 1 (Eq. 2): c_p = sum over
// its corners of (A_X(m_v) + A_Y(n_v)) d(m_v, n_v), with A the mixed vertex areas (the
// meshes' V are then required) and d the pair distances. normalize: divide the element
// costs by the largest one (c in [0, 1]).
int build_plan(const MeshIn& X, const MeshIn& Y, const float* d, const uint8_t* allowed,
               int split_chunk, int split_max_segments, int threads, Plan* out, std::string* err,
               bool normalize = true, int cost_model = 0);

}  // namespace disco
