// plan.cu -- variant choice, tiling and the comb launch.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <utility>
#include <vector>

#include "alnplot_internal.h"
#include "plan.h"

namespace ap {

namespace {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

const Variant *find_variant(int key_bits, int rows, int groups, int nu, int mu, int xrows)
{
    int count = 0;
    const Variant *t = variant_table(&count);
    for (int i = 0; i < count; ++i)
        if (t[i].key_bits == key_bits && t[i].rows == rows && t[i].groups == groups &&
            t[i].nu == nu && t[i].mu == mu && t[i].xrows == xrows)
            return &t[i];
    return nullptr;
}

// A variant can comb window w only if each thread's share of the strip's
// units (rows, or characters of a blow-up) fits its compiled rows and the
// rows left over fit its padding window: the kernels mask only the last
// PADU units of each thread as never-matching rows.
bool padding_ok(const Variant *v, int w)
{
    const int units = v->rows / v->nu;          // units per thread
    const int lo = w / v->groups;               // smallest share (even split)
    const int hi = (w + v->groups - 1) / v->groups;
    return hi <= units && units - lo <= v->padu;
}

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

bool choose_variant(int w, int nu, int mu, int want_groups, int64_t step, Plan *pl,
                    std::string *why, int want_lane_bits)
{
    const bool score = nu > 1;
    const int xrows = step > 1 ? 1 : 0;
    // key_bits: 7 (w <= 120), 8 (LCS, w <= 254: values fit a byte), 9 (LCS, 10-bit
    // lanes on request, 120 < w <= 480), else 15.
    int kbits = 0, rows = 0, groups = 0;
    auto rows_for = [&](int g, int unit, int lo, int hi) -> bool {
        // rows per thread for g threads: units (rows or pairs) rounded up to a
        // multiple of `unit`, at least lo; false if above hi
        int64_t r = std::max<int64_t>(lo, round_up(ceil_div(w, g), unit));
        if (r > hi) return false;
        groups = g;
        rows = (int)r;
        return true;
    };
    if (xrows) {
        // Vertical step: one x word per unit.  LCS: 7-bit keys up to w = 120,
        // full 8-bit keys up to 254, 16-bit lanes up to 512; {2,1,0}: 7-bit
        // pair keys up to 120, 16-bit lanes up to 256.
        if (!score && w <= 120) {
            kbits = 7;
            if (!rows_for(1, 8, 8, 64)) rows_for(2, 4, 36, 60);
        } else if (!score && w <= 254) {
            kbits = 8;
            if (want_groups == 4 || !rows_for(2, 64, 64, 64)) rows_for(4, 4, 32, 64);
        } else if (!score) {
            kbits = 15;
            if (want_groups != 8 && rows_for(4, 8, 16, 64)) {
            } else {
                rows_for(8, 8, 16, 64);
            }
        } else if (nu == 2 && mu == 1 && w <= 120) {
            kbits = 7;
            if (rows_for(4, 2, 2, 32)) rows *= 2;
        } else if (nu == 2 && mu == 1) {
            kbits = 15;
            if (rows_for(8, 4, 16, 32)) rows *= 2;
        }
    } else if (!score) {
        // A lane-format request (8, 10 or 16 bits) is honoured where that
        // format covers w: 8-bit lanes up to 254, 10-bit lanes for 257..480,
        // 16-bit lanes always; otherwise the default below.
        const bool want16 = want_lane_bits == 16 && w <= 512;
        const bool want10 = want_lane_bits == 10 && w > 120 && w <= 480;
        if (want16) {
            kbits = 15;
            if (want_groups == 2 || want_groups == 4 || want_groups == 8)
                rows_for(want_groups, 8, 16, want_groups == 4 ? 96 : 64);
            if (!rows)
                for (int g : {2, 4, 8})
                    if (rows_for(g, 8, 16, g == 4 ? 96 : 64)) break;
        } else if (want10) {
            kbits = 9;
            if (want_groups != 8) rows_for(4, 3, 33, 96);
            if (!rows) rows_for(8, 3, 33, 60);
        } else if (w <= 120) {
            kbits = 7;
            if (want_groups == 2) rows_for(2, 4, 16, 60);
            else if (want_groups == 4) rows_for(4, 4, 8, 32);
            if (!rows) rows_for(1, 4, 8, 120);
        } else if (w <= 240 || (want_lane_bits == 8 && w <= 254)) {
            // full 8-bit keys; above w = 240 (64 rows on 4 threads) 16-bit
            // lanes are faster: w = 254 285 ms against 339 ms
            kbits = 8;
            if (want_groups == 4 || !rows_for(2, 64, 64, 64)) rows_for(4, 4, 32, 64);
        } else {
            // 16-bit lanes (min/max cells): 4 threads up to 96 rows (w <= 384),
            // then 8.  Measured against 9-bit keys in 10-bit lanes on 100k DNA
            // plots: w = 272 326 vs 424 ms, w = 300 358 vs 451 ms, w = 384 407
            // vs 564 ms, w = 448 (8 threads) 552 vs 757 ms; 10-bit lanes stay
            // available on request.
            kbits = 15;
            if (want_groups == 2 || want_groups == 4 || want_groups == 8)
                rows_for(want_groups, 8, 16, want_groups == 4 ? 96 : 64);
            if (!rows)
                for (int g : {2, 4, 8})
                    if (rows_for(g, 8, 16, g == 4 ? 96 : 64)) break;
        }
    } else if (nu == 2 && mu == 1) {
        if (w <= 64) {
            kbits = 7;
            if (rows_for(1, 4, 4, 64)) rows *= 2;
        } else if (w <= 120) {
            kbits = 7;
            if (rows_for(2, 4, 36, 60)) rows *= 2;
        } else {
            // The window count and the value reach 2w, beyond 8-bit lanes.
            kbits = 15;
            if (rows_for(8, 4, 16, 32)) rows *= 2;
        }
    } else if (nu <= 4) {
        // {3 or 4, mu, 0}: 8-bit lanes while nu * w stays below 256 (w <= 32),
        // then 16-bit lanes on 8 threads (w <= 256).
        if (w <= 32) {
            kbits = 7;
            if (rows_for(1, 8, 8, 32)) rows *= nu;
        } else {
            kbits = 15;
            if (rows_for(8, 4, 4, 32)) rows *= nu;
        }
    } else {
        // {5..8, mu, 0}: 16-bit lanes on 8 threads, at most 128 rows a thread
        // (w <= 192 for nu = 5, 160 for 6, 128 for 7 and 8); one kernel per
        // nu and row count serves every mu (read at run time)
        kbits = 15;
        if (rows_for(8, 4, 4, 128 / nu / 4 * 4)) rows *= nu;
    }
    const Variant *v = (rows > 0) ? find_variant(kbits, rows, groups, nu, nu >= 5 ? -1 : mu, xrows) : nullptr;
    if (v && !padding_ok(v, w)) v = nullptr;
    if (!v && (want_groups > 0 || want_lane_bits > 0))   // a request no variant serves:
        return choose_variant(w, nu, mu, 0, step, pl, why, 0);   // the automatic choice
    if (!v) {
        if (why) {
            char buf[160];
            snprintf(buf, sizeof buf,
                     "no compiled comb variant for w=%d with scores {%d,%d,0} and step %lld", w, nu,
                     mu, (long long)step);
            *why = buf;
        }
        return false;
    }
    pl->v = v;
    pl->w = w;
    pl->step = step;
    pl->nu = nu;
    pl->mu = mu;
    pl->comb_rows = nu * w;
    pl->max_value = nu * w;
    // Exit ring and key range.  7-bit keys: the ring has next_pow2(2w + 2)
    // slots (32..128) and keys stay below the ring size, so the kernel's exit
    // counting needs no branch; the new key cycles through [w, ring - 1].
    // Full 8-bit keys: ring 256, keys in [w, 255].  9- and 15-bit keys find
    // exits by age: a valid exit at column c has age a < w and marks slot
    // c - a, and the slot of c - w is expired before column c's exits are
    // counted, so the live slots are the w columns c - w + 1 .. c and the
    // ring needs next_pow2(w) slots (w = 512: 16 KB a warp less than
    // next_pow2(w + 1), which had left room for one block per SM).
    if (v->key_bits == 7) {
        pl->ring = std::min(128, std::max(32, next_pow2(2 * w + 2)));
        pl->renorm = score ? (pl->ring - w) : (pl->ring - w) / 2;
    } else if (v->key_bits == 8) {
        pl->ring = 256;
        pl->renorm = score ? (256 - w) : (256 - w) / 2;
    } else if (v->key_bits == 9) {
        // keys cycle through [w, 511]; exits are found by age, as for 15-bit keys
        pl->ring = next_pow2(w);
        pl->renorm = (512 - w) / 2;
    } else {
        pl->ring = next_pow2(w);
        pl->renorm = score ? (32768 - w) : (32768 - w) / 2;
    }
    const int nlanes = v->lane_bits == 8 ? 4 : (v->lane_bits == 10 ? 3 : 2);
    pl->strips_per_warp = (32 / v->groups) * nlanes;
    const int ngrp = 32 / v->groups;
    pl->warp_words = pl->ring * ngrp + kOB * (ngrp + 1);
    if (has_tables(v->key_bits, v->groups, v->nu, v->xrows != 0)) pl->warp_words += tab_words(v->rows);
    if (has_tables_g(v->key_bits, v->groups, v->nu, v->xrows != 0))
        pl->warp_words += tabg_words(lane_strips(v->lane_bits), v->groups, v->rows);
    pl->smem = (size_t)kWarpsPerBlock * (size_t)pl->warp_words * 4u;
    return true;
}

static int resident_warps(const Plan &pl, int device)
{
    // Warps of this variant resident on the whole GPU at once (from the
    // occupancy calculator), or 8 per SM on a 152-SM part when no device is
    // available (host-only planning).
    int sms = 152, per_sm = 0;
    if (device >= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && v > 0)
            sms = v;
        else
            cudaGetLastError();
        if (pl.v && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &per_sm, (const void *)pl.v->fn, kWarpsPerBlock * 32, pl.smem) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
    }
    const int warps_per_sm = per_sm > 0 ? per_sm * kWarpsPerBlock : 8;
    return sms * warps_per_sm;
}

void tile_plan(Plan *pl, int64_t rows, int64_t cols, int64_t chunk_hint, int device)
{
    pl->rows = rows;
    pl->cols = cols;
    pl->nsg = ceil_div(rows, pl->strips_per_warp);
    int64_t chunk;
    if (chunk_hint > 0) {
        chunk = round_up(chunk_hint, kOB);
    } else {
        // All tiles of a launch take the same time, so the launch lasts
        // ceil(tiles / resident warps) rounds of one tile each, and a tile
        // combs its chunk plus the w - 1 warm-up columns (plus a few columns'
        // worth of setup).  Pick the chunk count that minimises
        //     ceil(nsg * nch / S) * (chunk(nch) + w - 1 + setup):
        // few chunks waste the last, partly filled round; many chunks pay
        // the warm-up again and again.
        const int64_t S = resident_warps(*pl, device);
        const int64_t setup = 8;
        const int64_t max_nch = std::max<int64_t>(1, ceil_div(std::max<int64_t>(cols, 1), kOB));
        int64_t best_nch = 1;
        double best = -1.0;
        for (int64_t nch = 1; nch <= max_nch; ++nch) {
            const int64_t ch = round_up(ceil_div(std::max<int64_t>(cols, 1), nch), kOB);
            if (ceil_div(std::max<int64_t>(cols, 1), ch) != nch) continue;   // same as a smaller count
            const int64_t rounds = ceil_div(pl->nsg * nch, S);
            const double cost = (double)rounds * (double)(ch + pl->w - 1 + setup);
            if (best < 0.0 || cost < best * (1.0 - 1e-9)) {
                best = cost;
                best_nch = nch;
            }
            if (rounds > 64 * ceil_div(pl->nsg, S) + 64) break;   // far past any useful split
        }
        chunk = round_up(ceil_div(std::max<int64_t>(cols, 1), best_nch), kOB);
    }
    chunk = std::min<int64_t>(chunk, round_up(std::max<int64_t>(cols, 1), kOB));
    chunk = std::min<int64_t>(chunk, 1LL << 30);   // tile-local indices are 32-bit
    pl->chunk = std::max<int64_t>(chunk, kOB);
    pl->nchunks = ceil_div(cols, pl->chunk);
    pl->ntiles = pl->nsg * pl->nchunks;
}

int64_t physical_cells(const Plan &pl)
{
    // every tile combs (its plot columns + w - 1) units of R rows x strips per warp
    const int64_t units = pl.cols + pl.nchunks * (int64_t)(pl.w - 1);
    const int64_t cols_phys = (int64_t)pl.nu * units;
    const int64_t comb_rows_padded = (int64_t)pl.v->rows * pl.v->groups;
    return pl.nsg * (int64_t)pl.strips_per_warp * cols_phys * comb_rows_padded;
}

#ifdef AP_DEBUG_BOUNDS
uint32_t *debug_flags()
{
    static std::mutex mu;
    static std::vector<std::pair<int, uint32_t *>> flags;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (auto &f : flags)
        if (f.first == dev) return f.second;
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t)) != cudaSuccess || cudaMemset(d, 0, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    flags.emplace_back(dev, d);
    return d;
}
#else
uint32_t *debug_flags() { return nullptr; }
#endif

void fill_params(const Plan &pl, const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                 void *out, int out_bytes, int64_t ld, CombParams *p)
{
    p->x = x;
    p->y = y;
    p->m = m;
    p->n = n;
    p->w = pl.w;
    p->renorm = pl.renorm;
    p->rows = pl.rows;
    p->cols = pl.cols;
    p->chunk = pl.chunk;
    p->nsg = pl.nsg;
    p->ntiles = pl.ntiles;
    p->tile0 = 0;
    p->out = out;
    p->ld = ld;
    p->out_bytes = out_bytes;
    const uintptr_t a = (uintptr_t)out;
    p->vec_ok = (out_bytes == 1) ? ((a % 4 == 0) && (ld % 4 == 0))
                                 : ((a % 8 == 0) && (ld % 4 == 0));
    p->ring = pl.ring;
    p->one = 1u;
    if (pl.v->lane_bits == 10) {
        // 10-bit lanes in bits 0-29: rows r = 1, 2 shift by 10r bits
        p->shmul[0] = p->shlo[0] = 1u;
        p->shmul[1] = 1u << 22;
        p->shlo[1] = 1u << 20;
        p->shmul[2] = 1u << 12;
        p->shlo[2] = 1u << 10;
        p->shmul[3] = p->shlo[3] = 0u;
    } else {
        p->shmul[0] = p->shlo[0] = 1u;
        p->shmul[1] = p->shlo[1] = 1u << 24;
        p->shmul[2] = p->shlo[2] = 1u << 16;
        p->shmul[3] = p->shlo[3] = 1u << 8;
    }
    p->spread_hi = 1u << 23;
    p->spread_lo = 0x3FFu;
    p->step = pl.step;
    p->warp_words = pl.warp_words;
    p->scale = (uint32_t)pl.scale;
    p->mu = pl.mu;
    const int t = plan_tables(pl);
    p->tab = t >= 2 ? t - 1 : 0;
    p->dbg = debug_flags();
}

int plan_tables(const Plan &pl)
{
    const Variant *v = pl.v;
    if (has_tables(v->key_bits, v->groups, v->nu, v->xrows != 0)) return 1;
    if (!has_tables_g(v->key_bits, v->groups, v->nu, v->xrows != 0)) return 0;
    const int mode = tabg_split_mode(pl.w, v->groups, v->rows, tabg_rpl(lane_strips(v->lane_bits)), v->padu);
    return mode ? 1 + mode : 0;
}

cudaError_t raise_smem_limit(const void *fn)
{
    // Raise a kernel's dynamic shared-memory limit once per device.
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == fn && d.second == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) done.emplace_back(fn, dev);
    return e;
}

cudaError_t launch_comb(const Plan &pl, const uint8_t *x, int64_t m, const uint8_t *y,
                        int64_t n, void *out, int out_bytes, int64_t ld, cudaStream_t stream)
{
    if (pl.ntiles == 0) return cudaSuccess;
    NvtxRange range("alnplot: comb launch");
    cudaError_t e0 = raise_smem_limit((const void *)pl.v->fn);
    if (e0 != cudaSuccess) return e0;
    CombParams p;
    fill_params(pl, x, m, y, n, out, out_bytes, ld, &p);
    const int64_t blocks = ceil_div(pl.ntiles, kWarpsPerBlock);
    // grid.x is limited to 2^31 - 1 blocks; split very large launches.
    const int64_t max_blocks = 1LL << 30;
    for (int64_t b0 = 0; b0 < blocks; b0 += max_blocks) {
        const int64_t nb = std::min(max_blocks, blocks - b0);
        p.tile0 = b0 * kWarpsPerBlock;
        pl.v->fn<<<(unsigned)nb, kWarpsPerBlock * 32, pl.smem, stream>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ap
