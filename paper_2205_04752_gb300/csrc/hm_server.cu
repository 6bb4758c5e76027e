// hm_server.cu -- a request loop over resident H-matrices.
//
// Matvec and solve requests on any of the server's matrices arrive over time
// (a trace replayed in real time, or all at once).  A scheduler thread admits
// them in arrival order as soon as a slot (worker thread with its own CUDA
// streams: matvec requests at the greatest stream priority, solves at the
// least) and enough device memory are free: every request's device
// footprint -- its vectors, the product workspace and, for a solve, the
// Krylov basis -- is carved out of one arena of fixed size by a first-fit
// allocator, so admission is by footprint.  Admitted requests run
// concurrently on their own streams, so their kernels overlap on the device
// while later requests keep arriving and being admitted (continuous
// batching at request granularity).  Arrivals that find the waiting queue
// full, or whose footprint exceeds the whole arena, are rejected.
//
// Each request runs exactly the kernels it would run alone (same forms, same
// number of right-hand sides per launch, its own workspace), so its result
// is bitwise the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hm_internal.h"

namespace {

using namespace hm;
using Clock = std::chrono::steady_clock;

constexpr size_t kGranule = 256;
size_t up(size_t b) { return (b + kGranule - 1) & ~(kGranule - 1); }

// first-fit allocator over [0, size) in 256-byte granules; host side only
class Arena {
  public:
    void init(size_t bytes)
    {
        free_.clear();
        size_ = bytes & ~(kGranule - 1);
        if (size_) free_[0] = size_;
        used_ = 0;
    }
    size_t alloc(size_t bytes)
    {
        bytes = up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                const size_t off = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem) free_[off + bytes] = rem;
                used_ += bytes;
                return off;
            }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

// counter-based uniform[-1, 1) inputs: splitmix64 of (seed, index)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void fill_uniform_kernel(double* __restrict__ x, int64_t n, uint32_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = splitmix64(((uint64_t)seed << 40) ^ (uint64_t)i);
        x[i] = 2.0 * ((double)(h >> 11) * 0x1.0p-53) - 1.0;
    }
}

}  // namespace

struct hm_server {
    std::vector<const hm_matrix*> mats;
    hm_server_params prm{};
    hm::Allocator alloc;
    hm::DevBuf arena_buf;
    int device = 0;
};

namespace {

struct Footprint {
    size_t total = 0;
    size_t x = 0, y = 0, ws = 0, scr = 0;  // offsets of the parts
};

Footprint footprint(const hm_server& S, const hm_request& q)
{
    const hm_matrix& H = *S.mats[(size_t)q.mesh];
    const size_t n = 3 * (size_t)H.M;
    Footprint f;
    if (q.kind == HM_REQ_MATVEC) {
        const size_t v = up((size_t)q.nrhs * n * 8);
        f.x = 0;
        f.y = v;
        f.scr = 2 * v;
        f.total = 2 * v + up(matvec_scratch_bytes(H, q.nrhs, S.prm.matvec_form));
    } else {
        const size_t v = up(n * 8);
        f.x = 0;
        f.y = v;
        f.ws = 2 * v;
        f.scr = f.ws + up(solve_workspace_bytes((int64_t)n, S.prm.restart));
        f.total = f.scr + up(std::max(matvec_scratch_bytes(H, 1, S.prm.inner_form),
                                      matvec_scratch_bytes(H, 1, S.prm.residual_form)));
    }
    return f;
}

struct Slot {
    std::thread th;
    bool has_job = false, done = false;
    int idx = -1;
    size_t off = 0, bytes = 0;
};

struct Run {
    Run(hm_server& s, const hm_request* q, hm_result* o) : S(s), reqs(q), out(o), t0(Clock::now()) {}
    hm_server& S;
    const hm_request* reqs;
    hm_result* out;
    std::mutex mu;
    std::condition_variable cv_work, cv_sched;
    std::vector<Slot> slots;
    bool stop = false;
    Clock::time_point t0;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    int execute(int idx, size_t off, cudaStream_t s, hm_result& r)
    {
        const hm_request& q = reqs[idx];
        const hm_matrix& H = *S.mats[(size_t)q.mesh];
        const int64_t n = 3 * H.M;
        const Footprint f = footprint(S, q);
        char* base = S.arena_buf.as<char>() + off;
        double* x = reinterpret_cast<double*>(base + f.x);
        double* y = reinterpret_cast<double*>(base + f.y);
        const int nv = q.kind == HM_REQ_MATVEC ? q.nrhs : 1;
        const size_t vbytes = (size_t)nv * (size_t)n * 8;
        int rc = HM_OK;
        if (q.x_host) {
            rc = cuda_check(cudaMemcpyAsync(x, q.x_host, vbytes, cudaMemcpyHostToDevice, s), "hm_server");
        } else {
            fill_uniform_kernel<<<256, 256, 0, s>>>(x, (int64_t)nv * n, (uint32_t)q.seed);
            rc = cuda_check(cudaGetLastError(), "hm_server");
        }
        if (rc) {
        } else if (q.kind == HM_REQ_MATVEC) {
            const Scratch scr = make_scratch(H, q.nrhs, S.prm.matvec_form, base + f.scr);
            rc = matvec_device_scratch(H, x, y, q.nrhs, n, S.prm.matvec_form, s, scr);
        } else {
            hm_solve_params p{};
            p.tol = q.tol > 0.0 ? q.tol : 1e-6;
            p.inner_tol = S.prm.inner_tol;
            p.inner_form = S.prm.inner_form;
            p.residual_form = S.prm.residual_form;
            p.restart = S.prm.restart;
            p.max_inner = S.prm.max_inner;
            rc = solve_check_params(&H, p);
            hm_solve_info info{};
            if (!rc) rc = solve_device(H, x, y, p, &info, s, base + f.ws, base + f.scr);
            r.iterations = info.iterations;
            r.rel_residual = info.rel_residual;
        }
        if ((!rc || rc == HM_ENOTCONV) && q.y_host) {
            const int e = cuda_check(cudaMemcpyAsync(q.y_host, y, vbytes, cudaMemcpyDeviceToHost, s), "hm_server");
            if (e) rc = e;
        }
        // nothing of this request may still run when its memory is released
        const int e = cuda_check(cudaStreamSynchronize(s), "hm_server");
        return e ? e : rc;
    }

    void worker(int w)
    {
        cudaSetDevice(S.device);
        // two streams per worker: matvec requests on the device's greatest
        // stream priority, solves on its least, so that the block scheduler
        // starts a matvec's CTAs ahead of those of solves that overlap it (the
        // kernels and their results are the same on either stream)
        int least = 0, greatest = 0;
        cudaStream_t s_mv = nullptr, s_sv = nullptr;
        bool have_stream = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
        have_stream = have_stream && cudaStreamCreateWithPriority(&s_mv, cudaStreamNonBlocking, greatest) == cudaSuccess;
        have_stream = have_stream && cudaStreamCreateWithPriority(&s_sv, cudaStreamNonBlocking, least) == cudaSuccess;
        for (;;) {
            int idx;
            size_t off;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || slots[(size_t)w].has_job; });
                if (stop && !slots[(size_t)w].has_job) break;
                idx = slots[(size_t)w].idx;
                off = slots[(size_t)w].off;
            }
            hm_result r{};
            cudaStream_t s = reqs[idx].kind == HM_REQ_MATVEC ? s_mv : s_sv;
            const int rc = have_stream ? execute(idx, off, s, r) : fail(HM_EDEVICE, "hm_server: no stream");
            const double t = now();
            {
                std::lock_guard<std::mutex> lk(mu);
                out[idx].status = rc;
                out[idx].iterations = r.iterations;
                out[idx].rel_residual = r.rel_residual;
                out[idx].done_s = t;
                slots[(size_t)w].has_job = false;
                slots[(size_t)w].done = true;
            }
            cv_sched.notify_one();
        }
        if (s_mv) cudaStreamDestroy(s_mv);
        if (s_sv) cudaStreamDestroy(s_sv);
    }
};

}  // namespace

extern "C" {

int hm_server_create(const hm_matrix* const* mats, int32_t nmat, const hm_server_params* prm, hm_server** out)
{
    if (!out) return fail(HM_EINVAL, "hm_server_create: NULL out");
    *out = nullptr;
    if (!mats || nmat < 1 || !prm) return fail(HM_EINVAL, "hm_server_create: need matrices and parameters");
    hm_server_params p = *prm;
    if (p.slots < 1 || p.slots > 64) return fail(HM_EINVAL, "hm_server_create: slots must lie in 1..64");
    if (p.queue_cap < 1) return fail(HM_EINVAL, "hm_server_create: queue_cap must be >= 1");
    if (p.budget_bytes < (int64_t)kGranule) return fail(HM_EINVAL, "hm_server_create: budget too small");
    if (p.restart <= 0) p.restart = 30;
    if (p.restart > 127) return fail(HM_EINVAL, "hm_server_create: restart above 127");
    if (p.inner_tol <= 0.0) p.inner_tol = 1e-3;
    if (p.solve_slots < 0 || p.solve_slots > p.slots)
        return fail(HM_EINVAL, "hm_server_create: solve_slots must lie in 0..slots");
    for (int32_t f : {p.matvec_form, p.inner_form, p.residual_form})
        if (f < HM_FP64 || f >= HM_NFORMS) return fail(HM_EINVAL, "hm_server_create: unknown form %d", f);
    for (int32_t m = 0; m < nmat; ++m) {
        const hm_matrix* H = mats[m];
        if (!H) return fail(HM_EINVAL, "hm_server_create: matrix %d is NULL", m);
        if (H->rect) return fail(HM_EINVAL, "hm_server_create: matrix %d: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm", m);
        for (int32_t f : {p.matvec_form, p.inner_form, p.residual_form})
            if (!H->packed[f]) return fail(HM_EINVAL, "hm_server_create: matrix %d has form %d not packed", m, f);
    }
    for (int32_t f : {p.matvec_form, p.inner_form, p.residual_form}) {
        int rc = product_prepare(f, nullptr);
        if (rc) return rc;
    }
    hm_server* S = new (std::nothrow) hm_server;
    if (!S) return fail(HM_ENOMEM, "hm_server_create: out of host memory");
    S->mats.assign(mats, mats + nmat);
    S->prm = p;
    S->alloc = mats[0]->alloc;
    S->alloc.stream = nullptr;
    cudaGetDevice(&S->device);
    S->arena_buf.bytes = (size_t)p.budget_bytes & ~(kGranule - 1);
    S->arena_buf.p = S->alloc.alloc(S->arena_buf.bytes);
    if (!S->arena_buf.p) {
        delete S;
        return fail(HM_ENOMEM, "hm_server_create: arena of %lld bytes", (long long)p.budget_bytes);
    }
    const int rc = cuda_check(cudaDeviceSynchronize(), "hm_server_create");
    if (rc) {
        S->alloc.release(S->arena_buf.p, S->arena_buf.bytes);
        delete S;
        return rc;
    }
    *out = S;
    return HM_OK;
}

int hm_server_footprint(const hm_server* S, const hm_request* q, int64_t* bytes)
{
    if (!S || !q || !bytes) return fail(HM_EINVAL, "hm_server_footprint: NULL argument");
    if (q->mesh < 0 || q->mesh >= (int32_t)S->mats.size()) return fail(HM_EINVAL, "hm_server_footprint: bad mesh");
    if (q->kind != HM_REQ_MATVEC && q->kind != HM_REQ_SOLVE) return fail(HM_EINVAL, "hm_server_footprint: bad kind");
    if (q->kind == HM_REQ_MATVEC && (q->nrhs < 1 || q->nrhs > 32))
        return fail(HM_EINVAL, "hm_server_footprint: nrhs outside 1..32");
    *bytes = (int64_t)up(footprint(*S, *q).total);
    return HM_OK;
}

int hm_server_run(hm_server* S, const hm_request* reqs, int32_t n, int32_t realtime, hm_result* out)
{
    if (!S || (n > 0 && (!reqs || !out)) || n < 0) return fail(HM_EINVAL, "hm_server_run: bad arguments");
    for (int32_t i = 0; i < n; ++i) {
        const hm_request& q = reqs[i];
        if (q.mesh < 0 || q.mesh >= (int32_t)S->mats.size())
            return fail(HM_EINVAL, "hm_server_run: request %d names mesh %d", i, q.mesh);
        if (q.kind != HM_REQ_MATVEC && q.kind != HM_REQ_SOLVE)
            return fail(HM_EINVAL, "hm_server_run: request %d has kind %d", i, q.kind);
        if (q.kind == HM_REQ_MATVEC && (q.nrhs < 1 || q.nrhs > 32))
            return fail(HM_EINVAL, "hm_server_run: request %d has nrhs %d outside 1..32", i, q.nrhs);
        if (realtime && i > 0 && q.arrival_s < reqs[i - 1].arrival_s)
            return fail(HM_EINVAL, "hm_server_run: arrivals must be sorted");
    }
    std::memset(out, 0, sizeof(hm_result) * (size_t)n);
    Arena arena;
    arena.init(S->arena_buf.bytes);
    Run R(*S, reqs, out);
    R.slots.resize((size_t)S->prm.slots);
    R.t0 = Clock::now();
    for (int w = 0; w < S->prm.slots; ++w) R.slots[(size_t)w].th = std::thread(&Run::worker, &R, w);

    std::deque<int> queue;
    int32_t next = 0, finished = 0;
    std::vector<int> idle;
    for (int w = S->prm.slots - 1; w >= 0; --w) idle.push_back(w);
    const int solve_cap = S->prm.solve_slots;
    int solves_running = 0;
    std::vector<size_t> fp((size_t)n);
    for (int32_t i = 0; i < n; ++i) fp[(size_t)i] = up(footprint(*S, reqs[i]).total);
    {
        std::unique_lock<std::mutex> lk(R.mu);
        while (finished < n) {
            const double t = R.now();
            // arrivals
            while (next < n && (!realtime || reqs[next].arrival_s <= t)) {
                hm_result& r = out[next];
                r.arrival_s = realtime ? reqs[next].arrival_s : 0.0;
                if (fp[(size_t)next] > arena.size() || (int32_t)queue.size() >= S->prm.queue_cap) {
                    r.status = HM_EBUSY;
                    r.start_s = r.done_s = t;
                    ++finished;
                } else {
                    queue.push_back(next);
                }
                ++next;
            }
            // completions
            for (size_t w = 0; w < R.slots.size(); ++w) {
                Slot& sl = R.slots[w];
                if (sl.done) {
                    sl.done = false;
                    if (reqs[sl.idx].kind == HM_REQ_SOLVE) --solves_running;
                    arena.release(sl.off, sl.bytes);
                    idle.push_back((int)w);
                    ++finished;
                }
            }
            // admission: each kind in arrival order, a free slot (a solve also
            // one of its solve_slots) and room in the arena; a solve that must
            // wait does not hold back the matvec requests behind it
            bool blocked[2] = {false, false};
            for (auto it = queue.begin(); it != queue.end() && !idle.empty();) {
                const int i = *it;
                const int kind = reqs[i].kind == HM_REQ_SOLVE ? 1 : 0;
                if (blocked[kind] || (kind == 1 && solve_cap > 0 && solves_running >= solve_cap)) {
                    blocked[kind] = true;
                    ++it;
                    if (blocked[0] && blocked[1]) break;
                    continue;
                }
                const size_t off = arena.alloc(fp[(size_t)i]);
                if (off == SIZE_MAX) break;  // memory: admit nothing out of order
                it = queue.erase(it);
                const int w = idle.back();
                idle.pop_back();
                Slot& sl = R.slots[(size_t)w];
                sl.idx = i;
                sl.off = off;
                sl.bytes = fp[(size_t)i];
                sl.has_job = true;
                if (kind == 1) ++solves_running;
                out[i].start_s = R.now();
                R.cv_work.notify_all();
            }
            if (finished >= n) break;
            double wait = 0.005;
            if (realtime && next < n) wait = std::min(wait, std::max(0.0, reqs[next].arrival_s - R.now()));
            R.cv_sched.wait_for(lk, std::chrono::duration<double>(wait));
        }
        R.stop = true;
    }
    R.cv_work.notify_all();
    for (auto& sl : R.slots) sl.th.join();
    // a device wait that ran out in any product invalidates the run
    for (size_t mi = 0; mi < S->mats.size(); ++mi) {
        const hm_matrix* H = S->mats[mi];
        int e[4] = {0, 0, 0, 0};  // flag, site, stage, CTA (as hm_check reports them)
        HM_CUDA(cudaMemcpy(e, H->d_err.p, sizeof e, cudaMemcpyDeviceToHost));
        if (e[0])
            return fail(HM_ETIMEOUT, "hm_server_run: a bounded device wait ran out (matrix %zu, site %d, stage %d, CTA %d)",
                        mi, e[1], e[2], e[3]);
    }
    return HM_OK;
}

void hm_server_destroy(hm_server* S)
{
    if (!S) return;
    cudaDeviceSynchronize();
    S->alloc.release(S->arena_buf.p, S->arena_buf.bytes);
    delete S;
}

}  // extern "C"
