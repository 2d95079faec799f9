// batch.cu -- many plot jobs as one CUDA graph of persistent comb kernels.
//
// The paper combs strips of one sequence pair.  A batch combs the strips of
// many pairs, with uneven lengths and window sizes, in one graph launch:
//   * jobs are grouped by comb variant (key width, rows per thread, threads
//     per strip group, score mode);
//   * every group gets a work list of tiles (job, strip group, column
//     chunk), most expensive first, and one persistent kernel whose warps
//     take tiles from an atomic counter until the list is empty;
//   * the groups' kernels run side by side on forked capture streams, so one
//     group's tail overlaps the others' work;
//   * an optional autotuner times candidate schedules (chunk length, threads
//     per strip) for every window class when the batch is created.
// Each tile is combed exactly as a plain launch combs it, so every job's plot
// is bit-identical to ap_alignment_plot's.
#include <sys/stat.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "alnplot_internal.h"
#include "plan.h"

namespace ap {
namespace {

struct Group {
    const Variant *v = nullptr;
    std::vector<int> jobs;       // indices into ap_batch::jobs
    int warp_words = 0;
    size_t smem = 0;
    int64_t ntiles = 0;
    BatchTile *d_tiles = nullptr;
    int blocks = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

// A tuned schedule of one window class: lane format (strips per register),
// threads per strip group and column chunk.
struct Schedule {
    int lane_bits = 0;
    int groups = 0;
    int64_t chunk = 0;
};

// Tuned schedules, keyed by the comb kernels' build digest, the device (name
// and SM count) and the window class (nu, mu, w).  Kept for the process and,
// unless AP_TUNE_CACHE=off, in a text file (AP_TUNE_CACHE, else
// $XDG_CACHE_HOME/alnplot/tune.txt or ~/.cache/alnplot/tune.txt), one line
// per class, so that later processes on the same kind of GPU skip the tuning.
#ifndef AP_KERNEL_DIGEST
#define AP_KERNEL_DIGEST "unversioned"
#endif
std::mutex g_tune_mu;
std::map<std::string, Schedule> g_tuned;
bool g_cache_loaded = false;

std::string tune_cache_path()
{
    const char *e = getenv("AP_TUNE_CACHE");
    if (e && *e) return strcmp(e, "off") == 0 ? std::string() : std::string(e);
    std::string dir;
    if (const char *x = getenv("XDG_CACHE_HOME")) dir = x;
    else if (const char *h = getenv("HOME")) dir = std::string(h) + "/.cache";
    else return std::string();
    mkdir(dir.c_str(), 0755);
    dir += "/alnplot";
    mkdir(dir.c_str(), 0755);
    return dir + "/tune.txt";
}

// Called with g_tune_mu held.
void load_tune_cache()
{
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char key[400];
        Schedule sc;
        long long chunk = 0;
        if (sscanf(line, "%399[^|]| %d %d %lld", key, &sc.lane_bits, &sc.groups, &chunk) == 4 && chunk > 0) {
            sc.chunk = chunk;
            g_tuned[key] = sc;
        }
    }
    fclose(f);
}

// Called with g_tune_mu held.
void store_tune_cache(const std::string &key, const Schedule &sc)
{
    g_tuned[key] = sc;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s| %d %d %lld\n", key.c_str(), sc.lane_bits, sc.groups, (long long)sc.chunk);
    fclose(f);
}

// The key also holds the class's size, as log2 buckets of its job count and
// its cells: the best schedule of a few small plots is not that of a
// thousand large ones.
std::string tune_key(int device, int nu, int mu, int w, int64_t njobs, double cells)
{
    cudaDeviceProp prop;
    std::string name = "unknown";
    int sms = 0;
    if (cudaGetDeviceProperties(&prop, std::max(0, device)) == cudaSuccess) {
        name = prop.name;
        sms = prop.multiProcessorCount;
    } else {
        cudaGetLastError();
    }
    for (char &c : name)
        if (c == ' ' || c == '|') c = '_';
    int jb = 0, cb = 0;
    while ((1LL << (jb + 1)) <= njobs) ++jb;
    while (cells >= 2.0 && cb < 80) {
        cells /= 2.0;
        ++cb;
    }
    char buf[400];
    snprintf(buf, sizeof buf, "%s %s sms=%d nu=%d mu=%d w=%d jobs=2^%d cells=2^%d ", AP_KERNEL_DIGEST,
             name.c_str(), sms, nu, mu, w, jb, cb);
    return buf;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Default batch chunk: long enough that the w - 1 warm-up columns cost at
// most ~6%, and no shorter than 2048 columns.
int64_t default_chunk(int w) { return std::max<int64_t>(2048, (16LL * w + 31) / 32 * 32); }

// Tiles of the jobs `idx` under `plans`, most expensive first.
std::vector<BatchTile> make_tiles(const std::vector<Plan> &plans, const std::vector<int> &idx)
{
    struct T {
        int64_t cost;
        BatchTile t;
    };
    std::vector<T> all;
    for (int j : idx) {
        const Plan &pl = plans[j];
        for (int64_t ch = 0; ch < pl.nchunks; ++ch) {
            const int64_t cols = std::min(pl.chunk, pl.cols - ch * pl.chunk);
            const int64_t units = cols + pl.w - 1;
            const int64_t cost = units * (int64_t)pl.v->rows * pl.nu;
            for (int64_t sg = 0; sg < pl.nsg; ++sg)
                all.push_back({cost, BatchTile{j, (int32_t)sg, (int32_t)ch, 0}});
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const T &a, const T &b) { return a.cost > b.cost; });
    std::vector<BatchTile> out(all.size());
    for (size_t i = 0; i < all.size(); ++i) out[i] = all[i].t;
    return out;
}

int resident_blocks(const Variant *v, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)v->batch_fn,
                                                      kWarpsPerBlock * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, per_sm) * std::max(1, sms);
}

}  // namespace
}  // namespace ap

using namespace ap;

struct ap_batch {
    int device = -1;
    std::vector<ap_job> jobs;
    std::vector<Plan> plans;
    std::vector<Group> groups;
    CombParams *d_params = nullptr;
    unsigned int *d_next = nullptr;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ap_batch_info info{};
};

namespace {

void release(ap_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &g : b->groups) {
        if (g.d_tiles) cudaFree(g.d_tiles);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->d_params) cudaFree(b->d_params);
    if (b->d_next) cudaFree(b->d_next);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

// Upload a group's tile list and size its persistent grid.
cudaError_t prepare_group(Group &g, const std::vector<Plan> &plans)
{
    g.warp_words = 0;
    for (int j : g.jobs) g.warp_words = std::max(g.warp_words, plans[j].warp_words);
    g.smem = (size_t)kWarpsPerBlock * (size_t)g.warp_words * 4u;
    std::vector<BatchTile> tiles = make_tiles(plans, g.jobs);
    g.ntiles = (int64_t)tiles.size();
    if (g.d_tiles) cudaFree(g.d_tiles);
    g.d_tiles = nullptr;
    if (g.ntiles == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&g.d_tiles, sizeof(BatchTile) * tiles.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(g.d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = raise_smem_limit((const void *)g.v->batch_fn);
    if (e != cudaSuccess) return e;
    g.blocks = (int)std::min<int64_t>(ceil_div(g.ntiles, kWarpsPerBlock),
                                      resident_blocks(g.v, g.smem));
    return cudaSuccess;
}

cudaError_t launch_group(const Group &g, const CombParams *d_params, unsigned int *counter,
                         cudaStream_t st)
{
    if (g.ntiles == 0) return cudaSuccess;
    BatchParams bp;
    bp.jobs = d_params;
    bp.tiles = g.d_tiles;
    bp.ntiles = g.ntiles;
    bp.next = counter;
    bp.warp_words = g.warp_words;
    g.v->batch_fn<<<g.blocks, kWarpsPerBlock * 32, g.smem, st>>>(bp);
    return cudaGetLastError();
}

cudaError_t upload_params(ap_batch *b)
{
    std::vector<CombParams> hp(b->jobs.size());
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        const ap_job &jb = b->jobs[j];
        fill_params(b->plans[j], jb.x, jb.m, jb.y, jb.n, jb.out, jb.out_elem_bytes, jb.ld, &hp[j]);
    }
    if (!b->d_params) {
        cudaError_t e = cudaMalloc(&b->d_params, sizeof(CombParams) * std::max<size_t>(1, hp.size()));
        if (e != cudaSuccess) return e;
    }
    if (hp.empty()) return cudaSuccess;
    return cudaMemcpy(b->d_params, hp.data(), sizeof(CombParams) * hp.size(), cudaMemcpyHostToDevice);
}

// Autotune one window class: try lane formats x threads per strip group x
// column chunks on a sample of the class's jobs (every fourth job of the
// class, in job order, when it has eight or more), timing one persistent
// launch each after one untimed launch; returns the fastest schedule.
ap_status tune_class(ap_batch *b, const std::vector<int> &idx, int nu, int w, Schedule *best,
                     double *tune_ms)
{
    // Candidate (lane bits, threads per strip group); 0 lane bits = the
    // default format for the window.  8-bit lanes always win over 16-bit
    // lanes up to w = 120 (twice the strips per instruction), so those are
    // not timed there.
    std::vector<std::pair<int, int>> cands;
    if (nu == 1) {
        std::vector<int> lbs;
        if (w <= 120) lbs = {8};
        else if (w <= 254) lbs = {8, 16};
        else if (w > 256 && w <= 480) lbs = {10, 16};
        else lbs = {16};
        for (int lb : lbs)
            for (int g : {1, 2, 4, 8}) cands.push_back({lb, g});
    } else {
        for (int g : {1, 2, 4, 8}) cands.push_back({0, g});
    }
    std::vector<int64_t> chunks_c = {1024, 4096, 16384};
    std::vector<int> sample;
    for (size_t k = 0; k < idx.size(); ++k)
        if (idx.size() < 8 || k % 4 == 0) sample.push_back(idx[k]);
    float best_ms = 1e30f;
    best->lane_bits = 0;
    best->groups = 0;
    best->chunk = default_chunk(w);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const auto t0 = std::chrono::steady_clock::now();
    ap_status st = AP_OK;
    for (auto [lb, gc] : cands) {
        for (int64_t cc : chunks_c) {
            if (cc < 4LL * w) continue;
            std::vector<Plan> saved;
            bool match = true;
            for (int j : sample) {
                saved.push_back(b->plans[j]);
                const ap_job &jb = b->jobs[j];
                ap_status s = plan_plot(jb.m, jb.n, jb.w, &jb.scores, gc, cc, &b->plans[j], 1, lb);
                if (s != AP_OK) {             // a request the planner cannot serve
                    match = false;
                    break;
                }
                const Variant *v = b->plans[j].v;
                match &= v->groups == gc && (lb == 0 || v->lane_bits == lb);
            }
            if (!match) {                  // no compiled variant for this request
                for (size_t k = 0; k < saved.size(); ++k) b->plans[sample[k]] = saved[k];
                continue;
            }
            Group g;
            g.v = b->plans[sample[0]].v;
            g.jobs = sample;
            cudaError_t e = upload_params(b);
            if (e == cudaSuccess) e = prepare_group(g, b->plans);
            float ms = 0;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned int), b->capture);
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->capture);
                if (e == cudaSuccess) e = launch_group(g, b->d_params, b->d_next, b->capture);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->capture);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            }
            if (g.d_tiles) cudaFree(g.d_tiles);
            for (size_t k = 0; k < sample.size(); ++k) b->plans[sample[k]] = saved[k];
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail_cuda(e, "batch autotune");
            }
            if (ms < best_ms) {
                best_ms = ms;
                best->lane_bits = lb;
                best->groups = gc;
                best->chunk = cc;
            }
        }
        if (st != AP_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tune_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // namespace

extern "C" {

ap_status ap_batch_create(const ap_job *jobs, int32_t njobs, const ap_batch_options *options,
                          ap_batch **out)
{
    if (!out) return fail(AP_E_INVAL, "ap_batch_create: null output pointer");
    *out = nullptr;
    if (njobs < 0 || (njobs > 0 && !jobs)) return fail(AP_E_INVAL, "ap_batch_create: bad job list");
    ap_batch_options opt{};
    if (options) opt = *options;
    if (opt.chunk < 0 || opt.lanes_per_strip < 0)
        return fail(AP_E_INVAL, "ap_batch_create: negative option");
    ap_batch *b = new ap_batch();
    b->device = current_device();

    // Validate and plan every job (jobs with an empty plot are dropped).
    for (int32_t j = 0; j < njobs; ++j) {
        const ap_job &jb = jobs[j];
        Plan pl;
        ap_status s = plan_plot(jb.m, jb.n, jb.w, &jb.scores, opt.lanes_per_strip,
                                opt.chunk > 0 ? opt.chunk : default_chunk(jb.w), &pl);
        if (s == AP_OK) s = check_output(pl, jb.x, jb.y, jb.out, jb.out_elem_bytes, jb.ld);
        if (s != AP_OK) {
            std::string msg = "job " + std::to_string(j) + ": " + ap_last_error();
            release(b);
            return fail(s, "%s", msg.c_str());
        }
        if (pl.ntiles == 0) continue;
        b->jobs.push_back(jb);
        b->plans.push_back(pl);
    }

    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned int) * 256);
    if (e != cudaSuccess) {
        release(b);
        return fail_cuda(e, "ap_batch_create");
    }

    // Autotune each window class (score mode, w), unless fixed by options.
    if (opt.autotune && opt.chunk == 0 && opt.lanes_per_strip == 0) {
        std::map<std::tuple<int, int, int>, std::vector<int>> classes;
        for (size_t j = 0; j < b->jobs.size(); ++j)
            classes[std::make_tuple(b->plans[j].nu, b->plans[j].mu, b->plans[j].w)].push_back((int)j);
        for (auto &kv : classes) {
            const int nu = std::get<0>(kv.first), mu = std::get<1>(kv.first), w = std::get<2>(kv.first);
            double cells = 0.0;
            for (int j : kv.second) cells += (double)b->plans[j].rows * b->plans[j].cols * w;
            const std::string key = tune_key(b->device, nu, mu, w, (int64_t)kv.second.size(), cells);
            Schedule best;
            bool cached = false;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                load_tune_cache();
                auto it = g_tuned.find(key);
                if (it != g_tuned.end()) {
                    best = it->second;
                    cached = true;
                }
            }
            if (!cached) {
                ap_status s = tune_class(b, kv.second, nu, w, &best, &b->info.tune_ms);
                if (s != AP_OK) {
                    release(b);
                    return s;
                }
                std::lock_guard<std::mutex> lk(g_tune_mu);
                store_tune_cache(key, best);
            }
            for (int j : kv.second) {
                const ap_job &jb = b->jobs[j];
                ap_status s = plan_plot(jb.m, jb.n, jb.w, &jb.scores, best.groups, best.chunk,
                                        &b->plans[j], 1, best.lane_bits);
                if (s != AP_OK) {
                    release(b);
                    return s;
                }
            }
        }
    }

    // Groups: one per comb variant, largest total work first.
    std::map<const Variant *, std::vector<int>> by_variant;
    for (size_t j = 0; j < b->jobs.size(); ++j) by_variant[b->plans[j].v].push_back((int)j);
    for (auto &kv : by_variant) {
        Group g;
        g.v = kv.first;
        g.jobs = kv.second;
        b->groups.push_back(g);
    }
    if (b->groups.size() > 256) {
        release(b);
        return fail(AP_E_UNSUPPORTED, "more than 256 comb variants in one batch");
    }
    e = upload_params(b);
    for (auto &g : b->groups) {
        if (e == cudaSuccess) e = prepare_group(g, b->plans);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    }
    std::stable_sort(b->groups.begin(), b->groups.end(),
                     [](const Group &a, const Group &c) { return a.ntiles > c.ntiles; });

    // Capture: reset the counters, fork one stream per group, join.
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned int) * b->groups.size(),
                                         b->capture);
        if (ce == cudaSuccess) ce = cudaEventRecord(b->fork, b->capture);
        for (size_t k = 0; k < b->groups.size() && ce == cudaSuccess; ++k) {
            Group &g = b->groups[k];
            ce = cudaStreamWaitEvent(g.stream, b->fork, 0);
            if (ce == cudaSuccess) ce = launch_group(g, b->d_params, b->d_next + k, g.stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(g.done, g.stream);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->capture, g.done, 0);
        }
        e = cudaStreamEndCapture(b->capture, &b->graph);
        if (ce != cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        release(b);
        return fail_cuda(e, "ap_batch_create");
    }

    b->info.groups = (int32_t)b->groups.size();
    b->info.jobs = (int32_t)b->jobs.size();
    for (auto &g : b->groups) b->info.tiles += g.ntiles;
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        const Plan &pl = b->plans[j];
        b->info.logical_cells += pl.rows * pl.cols * (int64_t)pl.w;
        b->info.physical_cells += physical_cells(pl);
    }
    *out = b;
    return AP_OK;
}

ap_status ap_batch_run(ap_batch *b, void *stream)
{
    if (!b) return fail(AP_E_INVAL, "ap_batch_run: null batch");
    if (!b->exec) return AP_OK;
    NvtxRange range("alnplot: batch graph launch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "ap_batch_run");
    return AP_OK;
}

ap_status ap_batch_get_info(const ap_batch *b, ap_batch_info *info)
{
    if (!b || !info) return fail(AP_E_INVAL, "ap_batch_get_info: null pointer");
    *info = b->info;
    return AP_OK;
}

ap_status ap_batch_destroy(ap_batch *b)
{
    release(b);
    return AP_OK;
}

}  // extern "C"
