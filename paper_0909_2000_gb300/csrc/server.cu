// server.cu -- a dot-plot server with admission by device memory and
// continuous batching across concurrent jobs.
//
// Requests (host sequences, window, threshold) are copied in and queued.  A
// scheduler thread admits them in arrival order, every job that fits a free
// slot and the device-memory budget (a job that does not fit yet does not
// block the ones behind it; one that has waited two seconds gets the next
// room).  An admitted job runs on its slot's own stream:
//   * copy x, y in and reset the running dot count;
//   * comb the plot band by band into the job's band buffer, each band
//     followed by its dot extraction (count, scan, write, appended in
//     row-major order);
//   * copy the count back; the scheduler then copies exactly that many dots
//     back and the job is done.
// The sequences and the partial plot (the current band) stay resident for
// the job's lifetime.  Jobs on different slots overlap on the device: one
// job's band kernels fill the SMs another job's kernels leave free.  A
// request that arrives while others run starts as soon as a slot and memory
// free up, and its result is the same as ap_alignment_dots's.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "alnplot_internal.h"
#include "plan.h"

namespace ap {
namespace {

using Clock = std::chrono::steady_clock;

// Plot band per job: a quarter of the budget's share per slot, within
// [32 MB, 512 MB].  Larger bands mean fewer launches per job and longer
// column chunks (less warm-up).  Measured on the Poisson serving workload
// (64 GiB, 16 slots): 128 MB bands gave 5.3e12 cells/s of capacity, 512 MB
// bands 5.6e12.
constexpr int64_t kBandMin = 32LL << 20, kBandMax = 512LL << 20;

int64_t band_bytes(int64_t budget, int slots)
{
    return std::min(kBandMax, std::max(kBandMin, budget / (4 * (int64_t)std::max(1, slots))));
}

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

struct Job {
    uint64_t ticket = 0;
    std::vector<uint8_t> x, y;
    int32_t w = 0;
    ap_scores scores{};
    int32_t threshold = 0;
    int64_t max_dots = 0;
    Plan plan;
    int64_t band_rows = 0, band_ld = 0;
    int elem = 1;
    // device layout (offsets from the job's allocation)
    int64_t off_y = 0, off_band = 0, off_counts = 0, off_offsets = 0, off_running = 0,
            off_dots = 0, dev_bytes = 0;
    enum State { QUEUED, RUNNING, DONE } state = QUEUED;
    ap_status status = AP_E_BUSY;
    bool cancelled = false;
    int phase = 0;
    int64_t count = 0;
    uint8_t *dev = nullptr;
    std::vector<ap_dot> result;
    Clock::time_point t_submit, t_done;
    std::string error;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Job *job = nullptr;
    uint8_t *pin_in = nullptr;
    int64_t pin_in_cap = 0;
    ap_dot *pin_out = nullptr;
    int64_t pin_out_cap = 0;
    int64_t *pin_count = nullptr;
};

void layout(Job &j, int64_t band)
{
    const Plan &pl = j.plan;
    j.elem = pl.max_value > 255 ? 2 : 1;
    j.band_ld = (pl.cols + 31) / 32 * 32;
    j.band_rows = band_rows_for(band / std::max<int64_t>(1, j.band_ld * j.elem),
                                pl.strips_per_warp, pl.rows);
    int64_t o = align256((int64_t)j.x.size());
    j.off_y = o;
    o += align256((int64_t)j.y.size());
    j.off_band = o;
    o += align256(j.band_rows * j.band_ld * j.elem);
    j.off_counts = o;
    o += align256(j.band_rows * 4);
    j.off_offsets = o;
    o += align256(j.band_rows * 8);
    j.off_running = o;
    o += 256;
    j.off_dots = o;
    o += align256(std::max<int64_t>(1, j.max_dots) * (int64_t)sizeof(ap_dot));
    j.dev_bytes = o;
}

}  // namespace
}  // namespace ap

using namespace ap;

struct ap_server {
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::condition_variable cv_work;
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, Job *> jobs;
    std::vector<Slot> slots;
    int64_t used = 0, peak = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread thread;
    int64_t submitted = 0, completed = 0, failed = 0, cells = 0;
    std::vector<double> latencies_ms;
};

namespace {

void finish(ap_server *s, Slot *slot, Job *j, ap_status st)
{
    // called with s->mu held
    if (j->cancelled) st = AP_E_CANCELLED;
    j->status = st;
    j->state = Job::DONE;
    j->t_done = Clock::now();
    if (slot) {
        if (j->dev) cudaFreeAsync(j->dev, slot->stream);
        j->dev = nullptr;
        s->used -= j->dev_bytes;
        slot->job = nullptr;
    }
    if (st == AP_OK || st == AP_E_OVERFLOW) {
        ++s->completed;
        s->cells += j->plan.rows * j->plan.cols * (int64_t)j->w;
        s->latencies_ms.push_back(
            std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count());
    } else {
        ++s->failed;
    }
    j->x.clear();
    j->x.shrink_to_fit();
    j->y.clear();
    j->y.shrink_to_fit();
    s->cv_done.notify_all();
}

cudaError_t grow_pinned(void **p, int64_t *cap, int64_t need)
{
    if (*cap >= need) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    const int64_t n = std::max<int64_t>(need, 1 << 20);
    cudaError_t e = cudaHostAlloc(p, (size_t)n, cudaHostAllocDefault);
    if (e == cudaSuccess) *cap = n;
    return e;
}

// Enqueue a job's whole GPU work on its slot's stream (phase 1).
cudaError_t start_job(ap_server *s, Slot &slot, Job &j)
{
    NvtxRange range("alnplot: server job start");
    cudaStream_t st = slot.stream;
    const int64_t m = (int64_t)j.x.size(), n = (int64_t)j.y.size();
    cudaError_t e = grow_pinned((void **)&slot.pin_in, &slot.pin_in_cap, m + n);
    if (e != cudaSuccess) return e;
    // The previous job on this slot has finished (its copies are complete).
    std::memcpy(slot.pin_in, j.x.data(), (size_t)m);
    std::memcpy(slot.pin_in + m, j.y.data(), (size_t)n);
    e = cudaMallocAsync((void **)&j.dev, (size_t)j.dev_bytes, st);
    if (e != cudaSuccess) return e;
    uint8_t *dx = j.dev, *dy = j.dev + j.off_y;
    void *band = j.dev + j.off_band;
    int32_t *counts = (int32_t *)(j.dev + j.off_counts);
    int64_t *offsets = (int64_t *)(j.dev + j.off_offsets);
    int64_t *running = (int64_t *)(j.dev + j.off_running);
    ap_dot *dots = (ap_dot *)(j.dev + j.off_dots);
    e = cudaMemcpyAsync(dx, slot.pin_in, (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, slot.pin_in + m, (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(running, 0, sizeof(int64_t), st);
    const Plan &pl = j.plan;
    for (int64_t r0 = 0; r0 < pl.rows && e == cudaSuccess; r0 += j.band_rows) {
        const int64_t br = std::min(j.band_rows, pl.rows - r0);
        Plan bp = pl;
        tile_plan(&bp, br, pl.cols, 0, s->device);
        e = launch_comb(bp, dx + r0, m - r0, dy, n, band, j.elem, j.band_ld, st);
        if (e == cudaSuccess)
            e = dots_pass(band, j.elem, br, pl.cols, j.band_ld, j.threshold, r0, dots, j.max_dots,
                          counts, offsets, running, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(slot.pin_count, running, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(slot.ev, st);
    j.phase = 1;
    return e;
}

// Admission policy: queued jobs are taken in arrival order, and every job
// that fits (a free slot, and its device memory within the budget) is
// admitted, so a large job at the head does not hold back the small ones
// behind it.  To keep large jobs from starving, once the oldest queued job
// has waited kAgeLimit it is admitted first: younger jobs are then only
// admitted while they leave room for it.
constexpr auto kAgeLimit = std::chrono::milliseconds(2000);

void scheduler(ap_server *s)
{
    cudaSetDevice(s->device);
    struct Start {
        Slot *slot;
        Job *job;
        cudaError_t err;
    };
    struct Done {
        Slot *slot;
        Job *job;
        int phase;          // the phase that finished: 1 comb and dots, 2 result copy
        cudaError_t err;
    };
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool busy = false;
        for (auto &sl : s->slots) busy |= sl.job != nullptr;
        if (s->stop && !busy) break;
        // ---- admission (under the lock: pick jobs, reserve slot and memory) ----
        std::vector<Start> starts;
        if (!s->stop) {
            const auto now = Clock::now();
            int64_t reserve = 0;     // memory held back for an aged head job
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                Job *j = *it;
                if (j->cancelled) {
                    it = s->queue.erase(it);
                    finish(s, nullptr, j, AP_E_CANCELLED);
                    continue;
                }
                if (j->plan.rows == 0 || j->plan.cols == 0) {   // empty plot: nothing to run
                    it = s->queue.erase(it);
                    j->count = 0;
                    finish(s, nullptr, j, AP_OK);
                    continue;
                }
                Slot *free_slot = nullptr;
                for (auto &sl : s->slots)
                    if (!sl.job) {
                        free_slot = &sl;
                        break;
                    }
                if (!free_slot) break;
                const bool aged = (now - j->t_submit) > kAgeLimit;
                if (s->used + reserve + j->dev_bytes > s->budget) {
                    if (aged && reserve == 0) reserve = j->dev_bytes;   // keep room for it
                    ++it;
                    continue;
                }
                it = s->queue.erase(it);
                j->state = Job::RUNNING;
                free_slot->job = j;
                s->used += j->dev_bytes;
                s->peak = std::max(s->peak, s->used);
                starts.push_back({free_slot, j, cudaSuccess});
            }
        }
        // ---- completions (event queries are cheap; the work is done unlocked) ----
        std::vector<Done> dones;
        for (auto &sl : s->slots) {
            Job *j = sl.job;
            if (!j || j->phase == 0) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            dones.push_back({&sl, j, j->phase, q});
        }
        if (starts.empty() && dones.empty()) {
            // Nothing to do: sleep briefly (GPU work in flight) or until a
            // submission arrives.
            s->cv_work.wait_for(lk, busy ? std::chrono::microseconds(50) : std::chrono::milliseconds(20));
            continue;
        }
        // ---- unlocked: pinned copies, allocations, enqueues, result copies ----
        lk.unlock();
        for (auto &st : starts) st.err = start_job(s, *st.slot, *st.job);
        for (auto &d : dones) {
            if (d.err != cudaSuccess) continue;
            Job *j = d.job;
            Slot &sl = *d.slot;
            if (d.phase == 1) {
                j->count = *sl.pin_count;
                const int64_t keep = std::min(j->count, j->max_dots);
                cudaError_t e = grow_pinned((void **)&sl.pin_out, &sl.pin_out_cap,
                                            keep * (int64_t)sizeof(ap_dot));
                if (e == cudaSuccess && keep > 0)
                    e = cudaMemcpyAsync(sl.pin_out, j->dev + j->off_dots, (size_t)keep * sizeof(ap_dot),
                                        cudaMemcpyDeviceToHost, sl.stream);
                if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
                d.err = e;
                j->phase = 2;
            } else {
                const int64_t keep = std::min(j->count, j->max_dots);
                j->result.assign(sl.pin_out, sl.pin_out + keep);
            }
        }
        lk.lock();
        // ---- publish (under the lock) ----
        for (auto &st : starts)
            if (st.err != cudaSuccess) {
                st.job->error = cudaGetErrorString(st.err);
                finish(s, st.slot, st.job, AP_E_CUDA);
            }
        for (auto &d : dones) {
            Job *j = d.job;
            if (d.err != cudaSuccess) {
                j->error = cudaGetErrorString(d.err);
                finish(s, d.slot, j, AP_E_CUDA);
            } else if (d.phase == 2) {
                if (j->cancelled) j->result.clear();
                finish(s, d.slot, j, j->count > j->max_dots ? AP_E_OVERFLOW : AP_OK);
            }
        }
    }
}

Job *find(ap_server *s, uint64_t t)
{
    auto it = s->jobs.find(t);
    return it == s->jobs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

ap_status ap_server_create(int64_t mem_budget, int32_t max_slots, ap_server **out)
{
    if (!out) return fail(AP_E_INVAL, "ap_server_create: null output pointer");
    *out = nullptr;
    if (mem_budget <= 0 || max_slots < 1 || max_slots > 64)
        return fail(AP_E_INVAL, "ap_server_create: need mem_budget > 0 and 1 <= max_slots <= 64");
    ap_server *s = new ap_server();
    s->device = std::max(0, current_device());
    s->budget = mem_budget;
    s->slots.resize(max_slots);
    for (auto &sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sl.pin_count, sizeof(int64_t), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            ap_server_destroy(s);
            return fail_cuda(e, "ap_server_create");
        }
    }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return AP_OK;
}

ap_status ap_server_submit(ap_server *s, const ap_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) return fail(AP_E_INVAL, "ap_server_submit: null pointer");
    if (r->m < 0 || r->n < 0 || (r->m > 0 && !r->x) || (r->n > 0 && !r->y))
        return fail(AP_E_INVAL, "ap_server_submit: bad sequence");
    if (r->max_dots < 0) return fail(AP_E_INVAL, "ap_server_submit: negative max_dots");
    Job *j = new Job();
    ap_status st = plan_plot(r->m, r->n, r->w, &r->scores, 0, 0, &j->plan);
    if (st != AP_OK) {
        delete j;
        return st;
    }
    j->x.assign(r->x, r->x + r->m);
    j->y.assign(r->y, r->y + r->n);
    j->w = r->w;
    j->scores = r->scores;
    j->threshold = r->threshold;
    j->max_dots = r->max_dots;
    layout(*j, band_bytes(s->budget, (int)s->slots.size()));
    if (j->dev_bytes > s->budget) {
        const long long need = (long long)j->dev_bytes;
        delete j;
        return fail(AP_E_NOMEM, "request needs %lld bytes of device memory, the budget is %lld",
                    need, (long long)s->budget);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete j;
        return fail(AP_E_CANCELLED, "server is shutting down");
    }
    j->ticket = s->next_ticket++;
    j->t_submit = Clock::now();
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    ++s->submitted;
    *ticket = j->ticket;
    s->cv_work.notify_all();
    return AP_OK;
}

ap_status ap_server_poll(ap_server *s, uint64_t ticket, ap_status *state)
{
    if (!s || !state) return fail(AP_E_INVAL, "ap_server_poll: null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    Job *j = find(s, ticket);
    if (!j) return fail(AP_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
    *state = j->state == Job::DONE ? j->status : AP_E_BUSY;
    return AP_OK;
}

ap_status ap_server_wait(ap_server *s, uint64_t ticket, int32_t timeout_ms)
{
    if (!s) return fail(AP_E_INVAL, "ap_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    Job *j = find(s, ticket);
    if (!j) return fail(AP_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
    auto done = [&] { return j->state == Job::DONE; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return fail(AP_E_TIMEOUT, "ticket %llu not finished after %d ms",
                    (unsigned long long)ticket, timeout_ms);
    }
    if (j->status != AP_OK)
        fail(j->status, "ticket %llu: %s", (unsigned long long)ticket,
             j->error.empty() ? ap_status_string(j->status) : j->error.c_str());
    return j->status;
}

ap_status ap_server_fetch(ap_server *s, uint64_t ticket, ap_dot *dots, int64_t cap,
                          int64_t *count)
{
    if (!s || !count || cap < 0 || (cap > 0 && !dots))
        return fail(AP_E_INVAL, "ap_server_fetch: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    Job *j = find(s, ticket);
    if (!j) return fail(AP_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (j->state != Job::DONE) return fail(AP_E_BUSY, "ticket %llu has not finished",
                                           (unsigned long long)ticket);
    const int64_t k = std::min<int64_t>(cap, (int64_t)j->result.size());
    if (k > 0) std::memcpy(dots, j->result.data(), (size_t)k * sizeof(ap_dot));
    *count = j->count;
    const ap_status st = j->status;
    s->jobs.erase(ticket);
    delete j;
    return st;
}

ap_status ap_server_cancel(ap_server *s, uint64_t ticket)
{
    if (!s) return fail(AP_E_INVAL, "ap_server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    Job *j = find(s, ticket);
    if (!j) return fail(AP_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (j->state == Job::QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), j), s->queue.end());
        j->cancelled = true;
        finish(s, nullptr, j, AP_E_CANCELLED);
    } else if (j->state == Job::RUNNING) {
        j->cancelled = true;
    }
    return AP_OK;
}

ap_status ap_server_get_stats(ap_server *s, ap_server_stats *out)
{
    if (!s || !out) return fail(AP_E_INVAL, "ap_server_get_stats: null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    ap_server_stats st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.queued = (int64_t)s->queue.size();
    for (auto &sl : s->slots) st.running += sl.job != nullptr;
    st.logical_cells = s->cells;
    st.peak_device_bytes = s->peak;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
            return v[i];
        };
        st.latency_p50_ms = pct(0.50);
        st.latency_p99_ms = pct(0.99);
        st.latency_max_ms = v.back();
    }
    *out = st;
    return AP_OK;
}

ap_status ap_server_destroy(ap_server *s)
{
    if (!s) return AP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        while (!s->queue.empty()) {
            Job *j = s->queue.front();
            s->queue.pop_front();
            finish(s, nullptr, j, AP_E_CANCELLED);
        }
        s->cv_work.notify_all();
    }
    if (s->thread.joinable()) s->thread.join();
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        if (sl.pin_count) cudaFreeHost(sl.pin_count);
    }
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return AP_OK;
}

}  // extern "C"
