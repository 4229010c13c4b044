// Autotuner (include/polymul.h, pm_autotune / pm_batch_autotune).
//
// The paper tunes its one parameter l once per machine by timing products
// with several values and keeping the fastest (Sec. 5, Sec. 7).  This
// library has more knobs -- the per-range strategy (direct-addressed slots
// or sort + reduce), the window size in slots (the tile), the number of
// groups per SM (the partition count), the slot accumulator, the weights
// of the group cost model, and for batches the term products per range and
// ranges per work item -- and tunes
// them the same way: every candidate runs on the caller's inputs, is timed
// with CUDA events on the caller's stream, and the fastest is kept for the
// problem's shape class.  pm_polymul called with default options looks the
// shape class up and uses the kept choice.
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "pm_common.cuh"

namespace pm {

// A shape class: kind, nvars, floor(log2) of n_f, n_g, the result bound
// min(n_f n_g, box) and the inputs' exponent box itself (so products with
// the same sizes but boxes of very different sparsity tune apart).
struct ShapeKey {
    int kind;
    u32 nvars;
    int lf, lg, lbound, lbox;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(kind, nvars, lf, lg, lbound, lbox) < std::tie(o.kind, o.nvars, o.lf, o.lg, o.lbound, o.lbox);
    }
};

static std::mutex g_tune_mu;
static std::map<ShapeKey, pm_options> g_tuned;

static int log2i(u64 x)
{
    int b = 0;
    while (x > 1) {
        x >>= 1;
        b++;
    }
    return b;
}

ShapeKey shape_key(int kind, u32 nvars, u64 nf, u64 ng, u64 bound, u64 raw_box)
{
    return ShapeKey{kind, nvars, log2i(nf), log2i(ng), log2i(bound), log2i(raw_box)};
}

// pm_out_bound's value and the inputs' exponent box (pm_api.cu)
int out_bound_and_box(const pm_packing *pk, const pm_terms_in *f, const pm_terms_in *g, u64 *bound, u64 *box,
                      cudaStream_t s);

// used by pm_polymul when its options are all defaults
u32 batch_range_chunk(u32 cw);  // pm_batch.cu

bool tuned_options(int kind, u32 nvars, u64 nf, u64 ng, u64 bound, u64 raw_box, pm_options &o)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(shape_key(kind, nvars, nf, ng, bound, raw_box));
    if (it == g_tuned.end()) return false;
    o = it->second;
    return true;
}

static void remember(const ShapeKey &k, const pm_options &o)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[k] = o;
}

}  // namespace pm

using namespace pm;

static float time_call(const pm_packing *pk, int kind, const pm_terms_in *f, const pm_terms_in *g, pm_terms_out *h,
                       const pm_options &o, cudaStream_t s, int reps, int *rc_out)
{
    pm_terms_out hh = *h;
    int rc = pm_polymul(pk, kind, f, g, &hh, &o, nullptr, s);  // warm-up (and validity)
    *rc_out = rc;
    if (rc != PM_OK) return -1.0f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r < reps; r++) {
        hh = *h;
        cudaEventRecord(a, s);
        rc = pm_polymul(pk, kind, f, g, &hh, &o, nullptr, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rc == PM_OK && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *h = hh;
    return best;
}

extern "C" int pm_autotune(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                           pm_terms_out *h, pm_options *best, pm_tune_report *report, void *stream)
{
    if (!pk || !f || !g || !h || !best) return PM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    u64 bound = 0, raw_box = 0;
    int rc = out_bound_and_box(pk, f, g, &bound, &raw_box, s);
    if (rc != PM_OK) return rc;

    std::vector<pm_options> cand;
    auto add = [&](int strategy, u32 slots, u32 gps, int acc, u32 chunk, u32 crow = 0, u32 cwin = 0, u32 grid_l = 0) {
        pm_options o;
        memset(&o, 0, sizeof(o));
        o.strategy = strategy;
        o.slots = slots;
        o.ranges_per_sm = gps;
        o.accumulator = acc;
        o.chunk = chunk;
        o.cost_row = crow;
        o.cost_window = cwin;
        o.grid_l = grid_l;
        cand.push_back(o);
    };
    // direct-addressed: partition count x tile x accumulator, and the
    // group cost model's weights
    for (u32 gps : {1u, 2u, 4u})
        for (u32 slots : {0u, 4096u, 12288u}) add(PM_STRATEGY_DIRECT, slots, gps, PM_ACC_AUTO, 0);
    add(PM_STRATEGY_DIRECT, 0, 1, PM_ACC_WIDE, 0);
    for (u32 gps : {1u, 2u}) {
        add(PM_STRATEGY_DIRECT, 0, gps, PM_ACC_AUTO, 0, 6, 12000);
        add(PM_STRATEGY_DIRECT, 0, gps, PM_ACC_AUTO, 0, 1, 8000);
    }
    // the Sec. 5 grid's l: the paper's 64, and a finer grid than the sizes'
    // choice, for the direct groups and the sort splitters
    add(PM_STRATEGY_DIRECT, 0, 1, PM_ACC_AUTO, 0, 0, 0, 64);
    add(PM_STRATEGY_DIRECT, 0, 1, PM_ACC_AUTO, 0, 0, 0, 1024);
    // sort + reduce: chunk sizes and grids; hashed windows
    for (u32 chunk : {2048u, 4096u}) add(PM_STRATEGY_SORT, 0, 0, PM_ACC_AUTO, chunk);
    for (u32 gl : {64u, 512u}) add(PM_STRATEGY_SORT, 0, 0, PM_ACC_AUTO, 4096, 0, 0, gl);
    add(PM_STRATEGY_HASH, 0, 0, PM_ACC_AUTO, 0);

    pm_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    int best_k = -1, first_err = PM_OK;
    float best_ms = 1e30f;
    for (size_t k = 0; k < cand.size() && k < PM_TUNE_MAX_CANDIDATES; k++) {
        int crc = PM_OK;
        // direct candidates on sparse boxes are refused by pm_polymul (box too large)
        const float ms = time_call(pk, coef_kind, f, g, h, cand[k], s, 2, &crc);
        rep.candidates[k] = cand[k];
        rep.ms[k] = crc == PM_OK ? ms : -1.0f;
        rep.count = (uint32_t)(k + 1);
        if (crc == PM_ECAPACITY) return crc;
        if (crc != PM_OK && first_err == PM_OK) first_err = crc;
        if (crc == PM_OK && ms < best_ms) {
            best_ms = ms;
            best_k = (int)k;
        }
    }
    if (best_k < 0) return first_err != PM_OK ? first_err : PM_EINVAL;
    *best = cand[best_k];
    rep.best = (uint32_t)best_k;
    if (report) *report = rep;
    remember(shape_key(coef_kind, pk->nvars, f->n, g->n, bound, raw_box), *best);
    return PM_OK;
}

extern "C" int pm_batch_autotune(const pm_batch_item *items, uint32_t count, pm_batch_options *best,
                                 pm_batch_tune_report *report, void *stream)
{
    if (!items || !count || !best) return PM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // tune on an evenly spaced sample of at most 256 items
    std::vector<pm_batch_item> sample;
    const uint32_t step = count > 256 ? count / 256 : 1;
    for (uint32_t k = 0; k < count && sample.size() < 256; k += step) sample.push_back(items[k]);
    pm_batch_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    float best_ms = 1e30f;
    int best_k = -1;
    int k = 0;
    // range sizes: fractions of the range kernel's shared-memory chunk,
    // which depends on the coefficient words of the whole batch (the
    // winner must be valid for every item, sampled or not)
    u32 cw = 1;
    for (uint32_t q = 0; q < count; q++)
        if (items[q].coef_kind == PM_COEF_I64_ACC128) cw = 2;
    const u32 ch = batch_range_chunk(cw);
    for (uint32_t target : {ch / 3, ch / 2, 3 * ch / 4, ch}) {
        for (uint32_t per : {8u, 16u, 64u}) {
            pm_batch_options o = {target, per};
            pm_batch_plan *pl = nullptr;
            int rc = pm_batch_plan_create(sample.data(), (uint32_t)sample.size(), &o, &pl, stream);
            if (rc != PM_OK) return rc;
            pm_batch_plan_run(pl, stream);  // warm-up
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            float ms_best = 1e30f;
            for (int r = 0; r < 2; r++) {
                cudaEventRecord(a, s);
                pm_batch_plan_run(pl, stream);
                cudaEventRecord(b, s);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                ms_best = ms < ms_best ? ms : ms_best;
            }
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            pm_batch_plan_destroy(pl);
            if (k < PM_TUNE_MAX_CANDIDATES) {
                rep.candidates[k] = o;
                rep.ms[k] = ms_best;
                rep.count = k + 1;
            }
            if (ms_best < best_ms) {
                best_ms = ms_best;
                best_k = k;
                *best = o;
            }
            k++;
        }
    }
    rep.best = (uint32_t)best_k;
    rep.sample = (uint32_t)sample.size();
    if (report) *report = rep;
    return PM_OK;
}
