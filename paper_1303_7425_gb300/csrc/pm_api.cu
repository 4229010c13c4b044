// Host driver and C-ABI entry points (include/polymul.h).
//
// pm_polymul runs Alg. 1 of the paper on one GPU: K-a canonical operands,
// K-b output ranges with balanced operation counts, K-c/K-d one CTA per range,
// K-e concatenation.  The host only reads sizes and status words between
// steps; every array the product touches is processed by the kernels.
#include <cstddef>
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "pm_bucket.cuh"
#include "pm_direct.cuh"
#include "pm_pack.cuh"
#include "pm_partition.cuh"
#include "pm_range.cuh"

namespace pm {

bool tuned_options(int kind, u32 nvars, u64 nf, u64 ng, u64 bound, u64 raw_box, pm_options &o);
int out_bound_and_box(const pm_packing *pk, const pm_terms_in *f, const pm_terms_in *g, u64 *bound, u64 *raw_box,
                      cudaStream_t s);

constexpr u32 DEFAULT_CHUNK = 4096;    // sort: term products per range
// bucket strategy: chosen automatically when its scratch -- a record and a
// result slot per term product, 32 bytes (mod p) or 56 bytes (int64) --
// stays within this many bytes
constexpr u64 BUCKET_MAX_BYTES = 32ull << 30;
constexpr u32 MAX_CHUNK = 4096;

// ---------------------------------------------------------------------------

static std::mutex g_dev_mu;
static int g_sm_count[64];
static bool g_pool_ready[64];

static void device_setup(Ctx &c)
{
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev < 64 && g_pool_ready[dev]) {
        c.sm_count = g_sm_count[dev];
        return;
    }
    int sms = 0;
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // keep freed scratch in this process's pool between calls
    cudaMemPool_t pool;
    PM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = ~0ull;
    PM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    if (dev < 64) {
        g_sm_count[dev] = sms;
        g_pool_ready[dev] = true;
    }
    c.sm_count = sms;
}

static void validate_packing(const pm_packing *pk)
{
    if (!pk || pk->nvars < 1 || pk->nvars > PM_MAX_VARS) throw Error(PM_EINVAL, "bad nvars");
    u32 sum = 0;
    for (u32 v = 0; v < pk->nvars; v++) {
        if (pk->field_bits[v] < 1 || pk->field_bits[v] > 32) throw Error(PM_EINVAL, "bad field width");
        sum += pk->field_bits[v];
    }
    if (sum > 64) throw Error(PM_EINVAL, "fields exceed 64 bits");
}

static void validate_terms(const pm_terms_in *t)
{
    if (!t) throw Error(PM_EINVAL, "null operand");
    if (t->n >= (1ull << 31)) throw Error(PM_EINVAL, "operand too large");
    if (t->n && (!t->exps || !t->coefs)) throw Error(PM_EINVAL, "null operand arrays");
}

static Layout base_layout(const pm_packing &pk)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    L.nv = pk.nvars;
    u32 s = 0;
    for (int v = (int)pk.nvars - 1; v >= 0; v--) {
        L.off[v] = s;
        L.width[v] = pk.field_bits[v];
        s += pk.field_bits[v];
    }
    return L;
}

// extents E_v = mf_v + mg_v + 1; strides of the mixed radix with x_1 most
// significant; returns the box size prod E_v (< 2^64 under the guard rule)
static u64 set_box(Layout &L, const u32 *mf, const u32 *mg)
{
    u64 stride = 1;
    for (int v = (int)L.nv - 1; v >= 0; v--) {
        L.extent[v] = (u64)mf[v] + mg[v] + 1;
        fastdiv_params(L.extent[v], L.dmag[v], L.dsh[v]);
        L.stride[v] = stride;
        stride *= L.extent[v];
    }
    return stride;
}

struct Small {  // host mirror of the small device block
    u32 status;
    u32 maxe_f[PM_MAX_VARS], maxe_g[PM_MAX_VARS];
    u32 pad;
    u64 count_f, count_g, maxabs_f, maxabs_g;
    u64 fl_f[2], fl_g[2];  // first and last canonical key of f and g
};

// A second stream for the steps on g that do not wait for f's (input
// maxima, canonical form, statistics, ranks): forked from the call's stream
// and joined back with events, so in a plan's capture they become parallel
// branches of the graph.  Its scratch is allocated on the side stream and
// freed there only after everything the call's stream enqueued, and the
// side stream is joined back once more after the frees.  One non-blocking
// stream per host thread and device.
static cudaStream_t side_stream()
{
    static thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(PM_ECUDA, "device index out of range");
    if (!streams[dev]) PM_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    return streams[dev];
}

struct Side {
    Ctx &main;
    Ctx c;
    std::unique_ptr<Scratch> S;
    cudaEvent_t ev = nullptr;
    Side(Ctx &m, ScratchMode sm) : main(m), c(m)
    {
        c.launches = 0;
        c.syncs = 0;
        c.s = side_stream();
        S.reset(new Scratch(c.s, sm));
        PM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    void fork()
    {
        PM_CUDA(cudaEventRecord(ev, main.s));
        PM_CUDA(cudaStreamWaitEvent(c.s, ev, 0));
    }
    void join()
    {
        PM_CUDA(cudaEventRecord(ev, c.s));
        PM_CUDA(cudaStreamWaitEvent(main.s, ev, 0));
        main.launches += c.launches;
        c.launches = 0;
    }
    ~Side()
    {
        // error paths too: no throwing here
        cudaEventRecord(ev, main.s);
        cudaStreamWaitEvent(c.s, ev, 0);
        S.reset();
        cudaEventRecord(ev, c.s);
        cudaStreamWaitEvent(main.s, ev, 0);
        cudaEventDestroy(ev);
    }
};

static void read_small(Ctx &c, Small &h, const Small *d)
{
    PM_CUDA(cudaMemcpyAsync(&h, d, sizeof(Small), cudaMemcpyDeviceToHost, c.s));
    c.sync();
}

// ---------------------------------------------------------------------------
// Plans (pm_plan_*): a product whose host decisions -- layout, operand
// sizes, partition sizes, strategy -- are recorded once and whose whole
// device path is then captured into one CUDA graph.  Every host decision
// of the call is a function of the small block read at its two host syncs,
// so a replay is exact whenever the small block it computes equals the
// recorded one; check kernels compare the two and, on any difference, set
// a flag at which the kernels that index by data return at entry.
// ---------------------------------------------------------------------------

constexpr u32 PLAN_MISMATCH = 1u, PLAN_CAPACITY = 2u;

struct PlanRec {
    enum Mode { DISCOVER, CAPTURE } mode = DISCOVER;
    Small snap[2];
    int nsnap = 0, ncap = 0;
    bool direct = false;      // the recorded call took the direct strategy
    Small *d_small = nullptr;  // the call's small block (plan-owned, persists)
    Small *d_snap = nullptr;   // device copies of snap[]
    u32 *d_flag = nullptr;     // PLAN_* bits of the last replay
    u64 *d_nout = nullptr;     // result size of the last replay
};

// Every word must be equal except the largest coefficient magnitudes
// (int64 kind; words [ma, ma + 4)), which may shrink: the int128 bound rule
// that passed for the recorded ones then holds too.
__global__ void k_plan_check(const u32 *__restrict__ cur, const u32 *__restrict__ rec, u32 words, u32 ma,
                             u32 *flag)
{
    u32 diff = 0;
    for (u32 k = threadIdx.x; k < words; k += blockDim.x)
        if (k < ma || k >= ma + 4) diff |= cur[k] ^ rec[k];
    if (threadIdx.x < 2) {
        const u64 c = (u64)cur[ma + 2 * threadIdx.x] | ((u64)cur[ma + 2 * threadIdx.x + 1] << 32);
        const u64 r = (u64)rec[ma + 2 * threadIdx.x] | ((u64)rec[ma + 2 * threadIdx.x + 1] << 32);
        if (c > r) diff = 1;
    }
    if (__syncthreads_or(diff != 0) && threadIdx.x == 0) atomicOr(flag, PLAN_MISMATCH);
}

// the small block after a step: read it (plain call; a plan's first call
// also records it), or, while a plan is captured, take the recorded one and
// enqueue the comparison with what the replay computes
static void fetch_small(Ctx &c, Small &h, const Small *d, PlanRec *rec)
{
    if (!rec || rec->mode == PlanRec::DISCOVER) {
        read_small(c, h, d);
        if (rec) {
            if (rec->nsnap >= 2) throw Error(PM_ECUDA, "plan: unexpected host sync");
            rec->snap[rec->nsnap++] = h;
        }
        return;
    }
    if (rec->ncap >= rec->nsnap) throw Error(PM_ECUDA, "plan: capture diverged from the recorded call");
    h = rec->snap[rec->ncap];
    static_assert(sizeof(Small) % 4 == 0, "small block in words");
    static_assert(offsetof(Small, maxabs_g) == offsetof(Small, maxabs_f) + 8, "maxabs words adjacent");
    k_plan_check<<<1, 128, 0, c.s>>>((const u32 *)d, (const u32 *)(rec->d_snap + rec->ncap), sizeof(Small) / 4,
                                     (u32)(offsetof(Small, maxabs_f) / 4), rec->d_flag);
    PM_LAUNCHED(c);
    rec->ncap++;
}

static u64 host_rank(const Layout &L, u64 key)
{
    u64 r = 0;
    for (u32 v = 0; v < L.nv; v++) r += ((key >> L.off[v]) & ((1ull << L.width[v]) - 1)) * L.stride[v];
    return r;
}

// The number of points of the rank box whose packed key is below `key`
// (any 64-bit value): lexicographic order with x_1 first equals rank order,
// so the output keys in [klo, khi) are the ranks [rank_below(klo),
// rank_below(khi)).  A digit at or past its extent means every box point
// with the same leading digits lies below.
static u64 rank_below(const Layout &L, u64 key)
{
    // bits above the fields (x_1's field ends the packed key) make the key
    // larger than every monomial of the box
    const u32 top = L.off[0] + L.width[0];
    if (top < 64 && (key >> top) != 0) return L.extent[0] * L.stride[0];
    u64 r = 0;
    for (u32 v = 0; v < L.nv; v++) {
        const u64 d = (key >> L.off[v]) & (L.width[v] >= 64 ? ~0ull : ((1ull << L.width[v]) - 1));
        if (d >= L.extent[v]) return r + L.extent[v] * L.stride[v];
        r += d * L.stride[v];
    }
    return r;
}

// A slice [lo, hi) of the output key space (pm_polymul_range,
// pm_shard_bounds); the whole space by default.
struct KeySlice {
    u64 lo = 0, hi = ~0ull;
    bool whole() const { return lo == 0 && hi == ~0ull; }
};

// What pm_shard_bounds asks of the call: after the canonical operands, the
// Alg. 2 split into nshards slices, and no product.
struct ShardQuery {
    u32 nshards = 0;
    u64 *bounds = nullptr;    // host, nshards + 1 keys
    u64 *products = nullptr;  // host, nshards term-product counts (optional)
};

// K-e for groups/ranges whose scratch slice starts at base[k] - base0
__global__ void k_compact_slices(const u64 *__restrict__ skey, const u64 *__restrict__ scoef,
                                 const u64 *__restrict__ base, u64 base0, const u64 *__restrict__ foff,
                                 const u64 *__restrict__ ucount, u32 nslices, u32 words, u64 *__restrict__ hkey,
                                 u64 *__restrict__ hcoef, u64 cap, u32 *plan_flag)
{
    // foff[nslices] is the result size: nothing is written past the
    // caller's capacity (a replayed plan reports it through plan_flag)
    if (foff[nslices] > cap) {
        if (plan_flag && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(plan_flag, PLAN_CAPACITY);
        return;
    }
    for (u32 k = blockIdx.x; k < nslices; k += gridDim.x) {
        const u64 src = base[k] - base0, dst = foff[k], n = ucount[k];
        for (u64 t = threadIdx.x; t < n; t += blockDim.x) {
            hkey[dst + t] = skey[src + t];
            for (u32 q = 0; q < words; q++) hcoef[words * (dst + t) + q] = scoef[words * (src + t) + q];
        }
    }
}

static int polymul_impl(const pm_packing *pk, int kind, const pm_terms_in *f, const pm_terms_in *g,
                        pm_terms_out *h, const pm_options *opt, pm_stats *st, cudaStream_t stream,
                        PlanRec *rec = nullptr, ScratchMode smode = ScratchMode(), KeySlice ks = KeySlice(),
                        ShardQuery *sq = nullptr)
{
    const bool capture = rec && rec->mode == PlanRec::CAPTURE;
    const u32 *abort = capture ? rec->d_flag : nullptr;
    validate_packing(pk);
    if (kind != PM_COEF_M61 && kind != PM_COEF_I64_ACC128 && kind != PM_COEF_I64_ACC192)
        throw Error(PM_EINVAL, "bad coefficient kind");
    validate_terms(f);
    validate_terms(g);
    if (!h) throw Error(PM_EINVAL, "null output");
    if (h->cap && (!h->keys || !h->coefs)) throw Error(PM_EINVAL, "null output arrays");
    h->n = 0;
    pm_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.chunk > MAX_CHUNK || o.strategy < 0 || o.strategy > 4 || o.accumulator < 0 || o.accumulator > 3 ||
        o.grid_l > 4096)
        throw Error(PM_EINVAL, "bad options");
    pm_stats stats;
    memset(&stats, 0, sizeof(stats));

    Ctx c;
    c.s = stream;
    device_setup(c);
    Scratch S(stream, smode);
    Small hs;
    Small *ds = rec ? rec->d_small : S.get<Small>(1);
    PM_CUDA(cudaMemsetAsync(ds, 0, sizeof(Small), c.s));
    if (capture) PM_CUDA(cudaMemsetAsync(rec->d_flag, 0, sizeof(u32), c.s));
    Side side(c, smode);  // g's steps; destroyed before S
    auto finish = [&](u64 n_out) {
        h->n = n_out;
        stats.n_out = n_out;
        if (st) {
            stats.kernel_launches = c.launches;
            stats.host_syncs = c.syncs;
            *st = stats;
        }
        return PM_OK;
    };

    // K-a (1): input guard bits and the raw exponent box            [sync 1]
    Layout L = base_layout(*pk);
    side.fork();
    input_maxima(c, *f, L, ds->maxe_f, &ds->status);
    input_maxima(side.c, *g, L, ds->maxe_g, &ds->status);
    side.join();
    fetch_small(c, hs, ds, rec);
    if (hs.status & ST_EXP_OVERFLOW) throw Error(PM_EEXP_OVERFLOW, "input exponent reaches its guard bit");
    if (f->n == 0 || g->n == 0) return finish(0);
    Layout raw = L;
    const u64 raw_box = set_box(raw, hs.maxe_f, hs.maxe_g);
    bool tuned = false;
    if (!opt || (!o.strategy && !o.slots && !o.chunk && !o.ranges_per_sm && !o.accumulator && !o.cost_row &&
                 !o.cost_window && !o.grid_l)) {
        // default options: use the autotuner's choice for this shape class
        const unsigned __int128 pr = (unsigned __int128)f->n * g->n;
        const u64 bound = pr < raw_box ? (u64)pr : raw_box;
        tuned = tuned_options(kind, L.nv, f->n, g->n, bound, raw_box, o);
    }

    // K-a (2): canonical operands, their maxima, extremes and sizes    [sync 2]
    Operand F, G;
    {
        // an operand whose own exponent box is small is canonicalised by a
        // scatter into that box, otherwise by a radix sort on its ranks
        const u32 zero[PM_MAX_VARS] = {0};
        Layout own_f = L, own_g = L;
        const u64 box_f = set_box(own_f, hs.maxe_f, zero);
        const u64 box_g = set_box(own_g, hs.maxe_g, zero);
        auto dense_ok = [](u64 box, u64 n) { return box <= (1ull << 26) && box <= 16 * n + 65536; };
        side.fork();
        if (dense_ok(box_f, f->n))
            canonicalize_dense(c, S, *f, own_f, box_f, kind, F, &ds->status, &ds->count_f, abort);
        else
            canonicalize(c, S, *f, raw, raw_box, kind, F, &ds->status, &ds->count_f);
        if (dense_ok(box_g, g->n))
            canonicalize_dense(side.c, *side.S, *g, own_g, box_g, kind, G, &ds->status, &ds->count_g, abort);
        else
            canonicalize(side.c, *side.S, *g, raw, raw_box, kind, G, &ds->status, &ds->count_g);
    }
    PM_CUDA(cudaMemsetAsync(ds->maxe_f, 0, sizeof(u32) * PM_MAX_VARS, c.s));
    PM_CUDA(cudaMemsetAsync(ds->maxe_g, 0, sizeof(u32) * PM_MAX_VARS, side.c.s));
    operand_stats(c, F, f->n, &ds->count_f, L, kind, ds->maxe_f, &ds->maxabs_f, ds->fl_f);
    operand_stats(side.c, G, g->n, &ds->count_g, L, kind, ds->maxe_g, &ds->maxabs_g, ds->fl_g);
    side.join();
    fetch_small(c, hs, ds, rec);
    if (hs.status & ST_COEF_BOUND) throw Error(PM_ECOEF_BOUND, "repeated input monomial leaves int64");
    F.n = hs.count_f;
    G.n = hs.count_g;
    stats.n_f = F.n;
    stats.n_g = G.n;
    if (F.n == 0 || G.n == 0) return finish(0);
    for (u32 v = 0; v < L.nv; v++)
        if ((u64)hs.maxe_f[v] + hs.maxe_g[v] >= (1ull << (L.width[v] - 1)))
            throw Error(PM_EEXP_OVERFLOW, "product exponent reaches its guard bit");
    if (kind == PM_COEF_I64_ACC128) {
        unsigned __int128 m = (unsigned __int128)hs.maxabs_f * hs.maxabs_g;
        unsigned __int128 lim = ((((unsigned __int128)1) << 127) - 1) / (F.n < G.n ? F.n : G.n);
        if (m > lim) throw Error(PM_ECOEF_BOUND, "int128 bound rule fails");
    }
    const u64 box = set_box(L, hs.maxe_f, hs.maxe_g);
    const u64 products = F.n * G.n;
    stats.term_products = products;
    stats.box = box;
    if (sq) {
        // Alg. 2: intervals from the Sec. 5 grid over the canonical
        // operands (about 64 per shard), their cumulative operation counts
        // O_k, and the split of the intervals into nshards groups
        const u64 kend = hs.fl_f[1] + hs.fl_g[1] + 1;
        u32 l = 1;
        while ((u64)(l + 1) * (l + 1) < 64ull * sq->nshards && l < 4096) l++;
        u32 ns = 0;
        const u64 *Sp = grid_splitters(c, S, F.key, (u32)F.n, G.key, (u32)G.n, l, kend, &ns);
        u64 *cnt = S.get<u64>(ns);
        count_below(c, F.key, (u32)F.n, G.key, (u32)G.n, Sp, ns, cnt);
        std::vector<u64> hS(ns), hc(ns);
        std::vector<u32> cut(sq->nshards + 1);
        PM_CUDA(cudaMemcpyAsync(hS.data(), Sp, (size_t)ns * 8, cudaMemcpyDeviceToHost, c.s));
        PM_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)ns * 8, cudaMemcpyDeviceToHost, c.s));
        c.sync();
        split_cumulative(hc.data(), ns, sq->nshards, cut.data());
        for (u32 m = 0; m <= sq->nshards; m++) sq->bounds[m] = hS[cut[m]];
        sq->bounds[0] = 0;
        sq->bounds[sq->nshards] = ~0ull;
        if (sq->products)
            for (u32 m = 0; m < sq->nshards; m++) sq->products[m] = hc[cut[m + 1]] - hc[cut[m]];
        if (sq->products) sq->products[sq->nshards - 1] = products - hc[cut[sq->nshards - 1]];
        return finish(0);
    }
    if (!ks.whole()) {
        // a slice of the output key space: nothing to do when it misses the
        // product's keys [first f + first g, last f + last g]
        const u64 klo = hs.fl_f[0] + hs.fl_g[0], kend = hs.fl_f[1] + hs.fl_g[1] + 1;
        if (ks.lo >= kend || ks.hi <= klo || ks.lo >= ks.hi) return finish(0);
    }
    const u32 words = kind == PM_COEF_M61 ? 1 : (kind == PM_COEF_I64_ACC192 ? 3 : 2);

    // strategy choice (autotuner defaults)
    int strategy = o.strategy;
    if (tuned && o.accumulator == PM_ACC_LIMBS && (F.n < G.n ? F.n : G.n) > 65537) o.accumulator = PM_ACC_AUTO;
    const u32 slots_max = direct_max_slots(kind, F.n < G.n ? F.n : G.n, o.accumulator);
    u32 slots = o.slots ? o.slots : slots_max;
    if (tuned && slots > slots_max) slots = slots_max;  // a class-mate's choice: keep it within this product's limits
    if (slots > slots_max) throw Error(PM_EINVAL, "slots exceed shared memory");
    const u32 chunk = o.chunk ? o.chunk : DEFAULT_CHUNK;
    // direct addressing's FindEdge table has a row of n_f words per window
    const u64 edge_words = ((box + slots - 1) / slots + (u64)c.sm_count * 4 + 1) * F.n;
    // the tuner's choice was made on another product of this shape class:
    // if this one cannot take the direct strategy, the automatic choice
    // below decides instead
    if (tuned && strategy == PM_STRATEGY_DIRECT && !(box < (1ull << 40) && edge_words <= (1ull << 30)))
        strategy = PM_STRATEGY_AUTO;
    if (strategy == PM_STRATEGY_AUTO) {
        // direct addressing pays when the rank box is not much larger than
        // the work (every slot of the box is cleared and scanned once) and
        // its windows' edge table stays within 2^30 words; a box up to 64
        // times the work takes hashed windows; sparser products the sort
        if (box <= 16 * products && box < (1ull << 40) && edge_words <= (1ull << 30))
            strategy = PM_STRATEGY_DIRECT;
        else if (box <= 64 * products)
            strategy = PM_STRATEGY_HASH;
        else if (kind != PM_COEF_I64_ACC192 && products >= (1ull << 20) &&
                 products <= BUCKET_MAX_BYTES / (kind == PM_COEF_M61 ? 32ull : 56ull))
            strategy = PM_STRATEGY_BUCKET;  // every product through the buckets
        else
            strategy = PM_STRATEGY_SORT;
    }
    if (strategy == PM_STRATEGY_BUCKET && kind == PM_COEF_I64_ACC192)
        throw Error(PM_EINVAL, "the bucket strategy takes the mod p and int128 kinds");
    if (strategy == PM_STRATEGY_DIRECT && box >= (1ull << 40))
        throw Error(PM_EINVAL, "exponent box too large for the direct strategy");
    stats.strategy = strategy;
    if (rec) rec->direct = strategy == PM_STRATEGY_DIRECT;
    // the sort strategy's partition refinement reads counts on the host
    if (capture && strategy != PM_STRATEGY_DIRECT) throw Error(PM_ECUDA, "plan: only the direct path is captured");


    u64 *okey, *ocoef, *ucount, *foff, *slice_base;
    u64 slice_base0;
    u32 nslices;
    // timing events (only when stats are asked for), destroyed on every
    // exit path
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    if (st)
        for (cudaEvent_t &x : ev.e) PM_CUDA(cudaEventCreate(&x));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1], k0 = ev.e[2], k1 = ev.e[3];

    if (strategy == PM_STRATEGY_HASH) {
        // hashed windows: rounds with host reads, then the result written
        // straight to h
        u32 *g32 = S.get<u32>(G.n);
        operand_ranks(c, F, L, nullptr);
        operand_ranks(c, G, L, g32);
        u64 lo = host_rank(L, hs.fl_f[0]) + host_rank(L, hs.fl_g[0]);
        u64 end = host_rank(L, hs.fl_f[1]) + host_rank(L, hs.fl_g[1]) + 1;
        if (!ks.whole()) {
            lo = std::max(lo, rank_below(L, ks.lo));
            end = std::min(end, rank_below(L, ks.hi));
            if (lo >= end) return finish(0);
        }
        HashInputs in;
        in.A = F.rank;
        in.Ac = F.coef;
        in.B = G.rank;
        in.Bc = G.coef;
        in.B32 = g32;
        in.na = (u32)F.n;
        in.nb = (u32)G.n;
        in.L = L;
        u32 rounds = 0;
        if (st) PM_CUDA(cudaEventRecord(e0, c.s));
        if (st) PM_CUDA(cudaEventRecord(k0, c.s));
        u64 windows = 0;
        const u64 n_out = hash_product(c, S, in, kind, o.accumulator, lo, end, products, (u64 *)h->keys,
                                       (u64 *)h->coefs, h->cap, &rounds, &windows);
        stats.n_ranges = windows;
        if (st) PM_CUDA(cudaEventRecord(k1, c.s));
        if (st) PM_CUDA(cudaEventRecord(e1, c.s));
        stats.refine_rounds = rounds;
        PM_CUDA(cudaMemcpyAsync(&hs.status, &ds->status, sizeof(u32), cudaMemcpyDeviceToHost, c.s));
        c.sync();
        if (st) {
            PM_CUDA(cudaEventElapsedTime(&stats.ms_range_step, e0, e1));
            PM_CUDA(cudaEventElapsedTime(&stats.ms_range_kernel, k0, k1));
        }
        if (hs.status & ST_INTERNAL) throw Error(PM_ECUDA, "internal consistency check failed");
        if (n_out > h->cap) {
            h->n = n_out;
            stats.n_out = n_out;
            if (st) {
                stats.kernel_launches = c.launches;
                stats.host_syncs = c.syncs;
                *st = stats;
            }
            return PM_ECAPACITY;
        }
        return finish(n_out);
    }

    if (strategy == PM_STRATEGY_BUCKET) {
        // every term product to a bucket of its key, each bucket sorted and
        // reduced in shared memory (pm_bucket.cu)
        u64 klo = hs.fl_f[0] + hs.fl_g[0], kend = hs.fl_f[1] + hs.fl_g[1] + 1;
        if (!ks.whole()) {
            klo = std::max(klo, ks.lo);
            kend = std::min(kend, ks.hi);
        }
        BucketInputs in;
        in.A = F.key;
        in.Ac = F.coef;
        in.B = G.key;
        in.Bc = G.coef;
        in.na = (u32)F.n;
        in.nb = (u32)G.n;
        in.A_last = hs.fl_f[1];
        in.B_last = hs.fl_g[1];
        if (st) PM_CUDA(cudaEventRecord(e0, c.s));
        if (st) PM_CUDA(cudaEventRecord(k0, c.s));
        const BucketSlices bs = bucket_product(c, S, in, kind, klo, kend, products);
        if (st) PM_CUDA(cudaEventRecord(k1, c.s));
        if (st) PM_CUDA(cudaEventRecord(e1, c.s));
        stats.n_ranges = bs.n;
        stats.refine_rounds = bs.big;
        okey = bs.key;
        ocoef = bs.coef;
        ucount = const_cast<u64 *>(bs.ucount);
        slice_base = const_cast<u64 *>(bs.base);
        slice_base0 = 0;
        nslices = (u32)bs.n;
    } else if (strategy == PM_STRATEGY_DIRECT) {
        // K-b: ranks, grid sample, groups (no host sync)
        u32 *g32 = S.get<u32>(G.n);
        u32 *f32 = box <= 0xFFFFFFFFull ? S.get<u32>(F.n) : nullptr;
        side.fork();
        operand_ranks(c, F, L, f32);
        operand_ranks(side.c, G, L, g32);
        side.join();
        u64 lo = host_rank(L, hs.fl_f[0]) + host_rank(L, hs.fl_g[0]);
        u64 end = host_rank(L, hs.fl_f[1]) + host_rank(L, hs.fl_g[1]) + 1;
        if (!ks.whole()) {
            lo = std::max(lo, rank_below(L, ks.lo));
            end = std::min(end, rank_below(L, ks.hi));
            if (lo >= end) return finish(0);
        }
        const u32 gps = o.ranges_per_sm ? o.ranges_per_sm : 1;
        u64 G64 = (u64)gps * c.sm_count;
        if (G64 > end - lo) G64 = end - lo;
        const u32 Gn = (u32)G64;
        // the Sec. 5 grid behind the cost histogram: about 4096 points per
        // group unless set (finer grids balanced the dense and 5-variable
        // products a few per cent better than 256 points per group)
        u32 l = 1;
        while ((u64)(l + 1) * (l + 1) < 4096ull * Gn && l < 4096) l++;
        if (o.grid_l) l = o.grid_l;
        const u32 crow = o.cost_row ? o.cost_row : 3u, cwin = o.cost_window ? o.cost_window : 23000u;
        const u64 *gb = direct_groups(c, S, F.rank, (u32)F.n, G.rank, (u32)G.n, lo, end, Gn, l, products, slots,
                                      crow, cwin);
        okey = S.get<u64>(end - lo);
        ocoef = S.get<u64>((end - lo) * words);
        DirectArgs a;
        memset(&a, 0, sizeof(a));
        a.A = F.rank;
        a.Ac = F.coef;
        a.B = G.rank;
        a.Bc = G.coef;
        a.B32 = g32;
        a.A32 = f32;
        a.na = (u32)F.n;
        a.nb = (u32)G.n;
        a.gb = gb;
        a.ngroups = Gn;
        a.lo = lo;
        a.okey = okey;
        a.ocoef = ocoef;
        a.L = L;
        a.abort = abort;
        if (st) PM_CUDA(cudaEventRecord(e0, c.s));
        launch_direct(c, S, a, slots, kind, o.accumulator, end, crow, cwin, k0, k1);
        if (st) PM_CUDA(cudaEventRecord(e1, c.s));
        stats.n_ranges = Gn;
        // the result slices are the windows, in rank order
        ucount = a.ucount;
        slice_base = const_cast<u64 *>(a.W);
        slice_base0 = lo;
        nslices = (u32)a.nwin_max;
    } else {
        // K-b: grid splitters, counts, refinement to the chunk capacity
        PartitionPlan plan;
        // the first splitters: the Sec. 5 grid with about four points per
        // chunk of term products, but at most the paper's l = 64, unless
        // set.  Finer first grids leave many ranges far below the chunk:
        // a 20000 x 20000 sparse 5-variable product took 568 ms with l =
        // 624 against 192 ms with 64 (the refinement splits the rest).
        double want = 4.0 * (double)products / chunk;
        u32 l = 1;
        while ((double)(l + 1) * (l + 1) < want && l < 64) l++;
        plan.grid_l = o.grid_l ? o.grid_l : l;
        plan.target = chunk;
        plan.hard_target = true;
        plan.max_rounds = 64;
        plan.key_lo = ks.lo;
        plan.key_hi = ks.hi;
        Ranges R = partition(c, S, F.key, (u32)F.n, G.key, (u32)G.n, plan);
        stats.n_ranges = R.n;
        stats.refine_rounds = R.rounds;
        RangeArgs a;
        memset(&a, 0, sizeof(a));
        a.fkey = F.key;
        a.fcoef = F.coef;
        a.gkey = G.key;
        a.gcoef = G.coef;
        a.na = (u32)F.n;
        a.nb = (u32)G.n;
        a.rlo = R.lo;
        a.rhi = R.hi;
        a.rO = R.O;
        a.boff = R.boff;
        a.nranges = R.n;
        okey = S.get<u64>(R.out_bound + 1);
        ocoef = S.get<u64>((R.out_bound + 1) * words);
        ucount = S.get<u64>(R.n + 1);
        a.okey = okey;
        a.ocoef = ocoef;
        a.ucount = ucount;
        a.L = L;
        a.status = &ds->status;
        if (st) PM_CUDA(cudaEventRecord(e0, c.s));
        if (st) PM_CUDA(cudaEventRecord(k0, c.s));
        if (R.n) launch_range_sort(c, a, chunk, kind, R.n);
        if (st) PM_CUDA(cudaEventRecord(k1, c.s));
        if (st) PM_CUDA(cudaEventRecord(e1, c.s));
        slice_base = R.boff;
        slice_base0 = 0;
        nslices = R.n;
    }

    // K-e: concatenate the slices in ascending order                  [sync 3]
    foff = S.get<u64>(nslices + 1);
    scan_exclusive_u64(c, S, ucount, foff, nslices);
    if (capture) {
        // no host read: the size goes to the plan, the capacity check to
        // the compaction kernel
        PM_CUDA(cudaMemcpyAsync(rec->d_nout, foff + nslices, sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
        if (nslices) {
            unsigned grid = nslices < 65535u ? nslices : 65535u;
            k_compact_slices<<<grid, 256, 0, c.s>>>(okey, ocoef, slice_base, slice_base0, foff, ucount, nslices, words,
                                                    (u64 *)h->keys, (u64 *)h->coefs, h->cap, rec->d_flag);
            PM_LAUNCHED(c);
        }
        return PM_OK;
    }
    u64 n_out = 0;
    PM_CUDA(cudaMemcpyAsync(&n_out, foff + nslices, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    PM_CUDA(cudaMemcpyAsync(&hs.status, &ds->status, sizeof(u32), cudaMemcpyDeviceToHost, c.s));
    c.sync();
    if (st) {
        PM_CUDA(cudaEventElapsedTime(&stats.ms_range_step, e0, e1));
        PM_CUDA(cudaEventElapsedTime(&stats.ms_range_kernel, k0, k1));
    }
    if (hs.status & ST_INTERNAL) throw Error(PM_ECUDA, "internal consistency check failed");
    stats.n_out = n_out;
    if (n_out > h->cap) {
        h->n = n_out;
        if (st) {
            stats.kernel_launches = c.launches;
            stats.host_syncs = c.syncs;
            *st = stats;
        }
        return PM_ECAPACITY;
    }
    if (nslices && n_out) {
        unsigned grid = nslices < 65535u ? nslices : 65535u;
        k_compact_slices<<<grid, 256, 0, c.s>>>(okey, ocoef, slice_base, slice_base0, foff, ucount, nslices, words,
                                                (u64 *)h->keys, (u64 *)h->coefs, h->cap, nullptr);
        PM_LAUNCHED(c);
    }
    return finish(n_out);
}

}  // namespace pm

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------

using namespace pm;

template <class F>
static int guarded(F &&fn)
{
    try {
        return fn();
    } catch (const Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return PM_ENOMEM;
    } catch (...) {
        return PM_ECUDA;
    }
}

extern "C" int pm_polymul(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                          pm_terms_out *h, const pm_options *opt, pm_stats *stats, void *stream)
{
    int rc = guarded([&] { return polymul_impl(pk, coef_kind, f, g, h, opt, stats, (cudaStream_t)stream); });
    if (rc != PM_OK && rc != PM_ECAPACITY && h) h->n = 0;
    return rc;
}

// The workspace a call on these inputs takes: the product runs once with
// pool scratch whose blocks are tallied, and writes no output (capacity 0).
// The hashed-window strategy may split a window more or less often from one
// run to the next (a window is split when a bounded hash-table probe runs
// out, and which probe does depends on the order of concurrent inserts), so
// its tally gets a margin of one quarter.
extern "C" int pm_workspace_size(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                                 const pm_options *opt, uint64_t *workspace_bytes, uint64_t *n_out, void *stream)
{
    if (!workspace_bytes) return PM_EINVAL;
    *workspace_bytes = 0;
    if (n_out) *n_out = 0;
    u64 tally = 0;
    pm_terms_out h;
    memset(&h, 0, sizeof(h));
    pm_stats st;
    memset(&st, 0, sizeof(st));
    ScratchMode sm;
    sm.tally = &tally;
    int rc = guarded([&] { return polymul_impl(pk, coef_kind, f, g, &h, opt, &st, (cudaStream_t)stream, nullptr, sm); });
    if (rc != PM_OK && rc != PM_ECAPACITY) return rc;
    if (st.strategy == PM_STRATEGY_HASH) tally += tally / 4;
    *workspace_bytes = tally;
    if (n_out) *n_out = h.n;
    return PM_OK;
}

extern "C" int pm_polymul_ws(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                             pm_terms_out *h, const pm_options *opt, pm_stats *stats, void *workspace,
                             uint64_t workspace_bytes, void *stream)
{
    if ((!workspace && workspace_bytes) || ((uintptr_t)workspace & 255u)) {
        if (h) h->n = 0;
        return PM_EINVAL;
    }
    Arena a;
    a.base = (char *)workspace;
    a.size = workspace_bytes;
    ScratchMode sm;
    sm.arena = &a;
    int rc = guarded([&] { return polymul_impl(pk, coef_kind, f, g, h, opt, stats, (cudaStream_t)stream, nullptr, sm); });
    if (rc != PM_OK && rc != PM_ECAPACITY && h) h->n = 0;
    return rc;
}

extern "C" int pm_polymul_range(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                                uint64_t key_lo, uint64_t key_hi, pm_terms_out *h, const pm_options *opt,
                                pm_stats *stats, void *stream)
{
    KeySlice ks;
    ks.lo = key_lo;
    ks.hi = key_hi;
    int rc = guarded([&] {
        return polymul_impl(pk, coef_kind, f, g, h, opt, stats, (cudaStream_t)stream, nullptr, ScratchMode(), ks);
    });
    if (rc != PM_OK && rc != PM_ECAPACITY && h) h->n = 0;
    return rc;
}

extern "C" int pm_shard_bounds(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                               uint32_t nshards, uint64_t *bounds, uint64_t *products, void *stream)
{
    if (nshards < 1 || nshards > 65536 || !bounds) return PM_EINVAL;
    for (u32 m = 0; m <= nshards; m++) bounds[m] = m == nshards ? ~0ull : 0ull;
    if (products)
        for (u32 m = 0; m < nshards; m++) products[m] = 0;
    ShardQuery sq;
    sq.nshards = nshards;
    sq.bounds = (u64 *)bounds;
    sq.products = (u64 *)products;
    pm_terms_out h;
    memset(&h, 0, sizeof(h));
    return guarded([&] {
        return polymul_impl(pk, coef_kind, f, g, &h, nullptr, nullptr, (cudaStream_t)stream, nullptr, ScratchMode(),
                            KeySlice(), &sq);
    });
}

extern "C" int pm_split_cumulative(const uint64_t *cum, uint32_t n, uint32_t nshards, uint32_t *cut)
{
    if (!cum || !cut || nshards < 1 || n < 1) return PM_EINVAL;
    for (u32 k = 1; k < n; k++)
        if (cum[k] < cum[k - 1]) return PM_EINVAL;
    split_cumulative((const u64 *)cum, n, nshards, cut);
    return PM_OK;
}

int pm::out_bound_and_box(const pm_packing *pk, const pm_terms_in *f, const pm_terms_in *g, u64 *bound,
                          u64 *raw_box, cudaStream_t s)
{
    return guarded([&] {
        validate_packing(pk);
        validate_terms(f);
        validate_terms(g);
        if (!bound) throw Error(PM_EINVAL, "null bound");
        *bound = 0;
        if (raw_box) *raw_box = 0;
        if (f->n == 0 || g->n == 0) return PM_OK;
        Ctx c;
        c.s = s;
        device_setup(c);
        Scratch S(c.s);
        Small hs;
        Small *ds = S.get<Small>(1);
        PM_CUDA(cudaMemsetAsync(ds, 0, sizeof(Small), c.s));
        Layout L = base_layout(*pk);
        input_maxima(c, *f, L, ds->maxe_f, &ds->status);
        input_maxima(c, *g, L, ds->maxe_g, &ds->status);
        read_small(c, hs, ds);
        if (hs.status & ST_EXP_OVERFLOW) throw Error(PM_EEXP_OVERFLOW, "input exponent reaches its guard bit");
        u64 box = set_box(L, hs.maxe_f, hs.maxe_g);
        unsigned __int128 prod = (unsigned __int128)f->n * g->n;
        *bound = prod < box ? (u64)prod : box;
        if (raw_box) *raw_box = box;
        return PM_OK;
    });
}

extern "C" int pm_out_bound(const pm_packing *pk, const pm_terms_in *f, const pm_terms_in *g, uint64_t *bound,
                            void *stream)
{
    u64 b = 0;
    const int rc = out_bound_and_box(pk, f, g, &b, nullptr, (cudaStream_t)stream);
    if (bound) *bound = b;
    return rc;
}

extern "C" int pm_grid(const uint64_t *alpha, uint64_t na, const uint64_t *beta, uint64_t nb, uint32_t l,
                       uint64_t *splitters, uint64_t cap, uint64_t *n_out, void *stream)
{
    return guarded([&] {
        if (!n_out) throw Error(PM_EINVAL, "null n_out");
        *n_out = 0;
        if (l < 1 || l > 4096) throw Error(PM_EINVAL, "l outside 1..4096");
        if (na >= (1ull << 31) || nb >= (1ull << 31)) throw Error(PM_EINVAL, "operand too large");
        if (na == 0 || nb == 0) return PM_OK;
        if (!alpha || !beta) throw Error(PM_EINVAL, "null keys");
        if (cap && !splitters) throw Error(PM_EINVAL, "null output");
        Ctx c;
        c.s = (cudaStream_t)stream;
        device_setup(c);
        Scratch S(c.s);
        u64 ext[2];
        PM_CUDA(cudaMemcpyAsync(&ext[0], alpha + na - 1, 8, cudaMemcpyDeviceToHost, c.s));
        PM_CUDA(cudaMemcpyAsync(&ext[1], beta + nb - 1, 8, cudaMemcpyDeviceToHost, c.s));
        c.sync();
        const u64 end = ext[0] + ext[1] + 1;
        u32 ns = 0;
        const u64 *Sp = grid_splitters(c, S, (const u64 *)alpha, (u32)na, (const u64 *)beta, (u32)nb, l, end, &ns);
        *n_out = ns;
        if (ns > cap) return PM_ECAPACITY;
        PM_CUDA(cudaMemcpyAsync(splitters, Sp, (size_t)ns * 8, cudaMemcpyDeviceToDevice, c.s));
        c.sync();
        return PM_OK;
    });
}

extern "C" int pm_unpack(const pm_packing *pk, const uint64_t *keys, uint64_t n, uint32_t *exps, void *stream)
{
    return guarded([&] {
        validate_packing(pk);
        if (n && (!keys || !exps)) throw Error(PM_EINVAL, "null arrays");
        Ctx c;
        c.s = (cudaStream_t)stream;
        unpack_keys(c, (const u64 *)keys, n, base_layout(*pk), exps);
        return PM_OK;
    });
}

extern "C" int pm_pack(const pm_packing *pk, const uint32_t *exps, uint64_t n, uint64_t *keys, void *stream)
{
    return guarded([&] {
        validate_packing(pk);
        if (n && (!keys || !exps)) throw Error(PM_EINVAL, "null arrays");
        if (n == 0) return PM_OK;
        Ctx c;
        c.s = (cudaStream_t)stream;
        Scratch S(c.s);
        u32 *st = S.get<u32>(1);
        PM_CUDA(cudaMemsetAsync(st, 0, sizeof(u32), c.s));
        pack_keys(c, exps, n, base_layout(*pk), (u64 *)keys, st);
        u32 hst = 0;
        PM_CUDA(cudaMemcpyAsync(&hst, st, sizeof(u32), cudaMemcpyDeviceToHost, c.s));
        c.sync();
        if (hst & ST_EXP_OVERFLOW) throw Error(PM_EEXP_OVERFLOW, "exponent reaches its guard bit");
        return PM_OK;
    });
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------

struct pm_plan {
    PlanRec rec;
    pm_packing pk;
    int kind;
    pm_terms_in f, g;
    pm_terms_out h;
    pm_options opt;
    bool has_opt = false;
    bool captured = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    u32 *host = nullptr;   // pinned: flag, status, n_out (2 words)
    int last_rc = PM_OK;   // plain (not captured) plans: result of the last run
    u64 last_n = 0;
};

static void plan_free(pm_plan *p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->rec.d_small) cudaFree(p->rec.d_small);
    if (p->host) cudaFreeHost(p->host);
    delete p;
}

extern "C" int pm_plan_create(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                              pm_terms_out *h, const pm_options *opt, pm_plan **plan, void *stream)
{
    if (!plan) return PM_EINVAL;
    *plan = nullptr;
    pm_plan *p = new (std::nothrow) pm_plan;
    if (!p) return PM_ENOMEM;
    int rc = guarded([&] {
        if (!pk || !f || !g || !h) throw Error(PM_EINVAL, "null argument");
        p->pk = *pk;
        p->kind = coef_kind;
        p->f = *f;
        p->g = *g;
        p->h = *h;
        p->has_opt = opt != nullptr;
        if (opt) p->opt = *opt;
        // one device block: the call's small block, the two recorded
        // snapshots, the flag and the result size
        const size_t bytes = 3 * sizeof(Small) + 16;
        void *d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw Error(PM_ENOMEM, "plan block");
        }
        p->rec.d_small = (Small *)d;
        p->rec.d_snap = p->rec.d_small + 1;
        p->rec.d_flag = (u32 *)(p->rec.d_small + 3);
        p->rec.d_nout = (u64 *)((char *)d + 3 * sizeof(Small) + 8);
        PM_CUDA(cudaMemset(d, 0, bytes));
        PM_CUDA(cudaMallocHost((void **)&p->host, 16));
        // the recorded call: a plain product that also fills h
        cudaStream_t s = (cudaStream_t)stream;
        p->rec.mode = PlanRec::DISCOVER;
        int r = polymul_impl(pk, coef_kind, f, g, h, opt, nullptr, s, &p->rec);
        if (r != PM_OK) return r;
        p->last_n = h->n;
        if (!p->rec.direct || p->rec.nsnap != 2) return PM_OK;  // runs as plain calls
        PM_CUDA(cudaMemcpy(p->rec.d_snap, p->rec.snap, 2 * sizeof(Small), cudaMemcpyHostToDevice));
        // capture on a stream of our own (the caller's may be the legacy
        // default stream, which cannot be captured)
        cudaStream_t cs;
        PM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        p->rec.mode = PlanRec::CAPTURE;
        p->rec.ncap = 0;
        pm_terms_out hh = *h;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            throw Error(PM_ECUDA, "begin capture");
        }
        int crc = PM_OK;
        try {
            crc = polymul_impl(pk, coef_kind, f, g, &hh, opt, nullptr, cs, &p->rec);
        } catch (const Error &err) {
            crc = err.code;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (crc != PM_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw Error(crc != PM_OK ? crc : PM_ECUDA, "capture");
        }
        p->graph = graph;
        PM_CUDA(cudaGraphInstantiate(&p->exec, graph, 0));
        p->captured = true;
        return PM_OK;
    });
    if (rc != PM_OK) {
        plan_free(p);
        return rc;
    }
    *plan = p;
    return PM_OK;
}

extern "C" int pm_plan_run(pm_plan *p, void *stream)
{
    if (!p) return PM_EINVAL;
    if (p->captured) {
        cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return PM_ECUDA;
        }
        return PM_OK;
    }
    // not captured (sort strategy or an empty product): a plain call
    pm_terms_out hh = p->h;
    p->last_rc = pm_polymul(&p->pk, p->kind, &p->f, &p->g, &hh, p->has_opt ? &p->opt : nullptr, nullptr, stream);
    p->last_n = hh.n;
    return p->last_rc == PM_ECAPACITY ? PM_OK : p->last_rc;
}

extern "C" int pm_plan_finish(pm_plan *p, uint64_t *n_out, void *stream)
{
    if (!p) return PM_EINVAL;
    if (!p->captured) {
        if (n_out) *n_out = p->last_n;
        return p->last_rc;
    }
    return guarded([&] {
        cudaStream_t s = (cudaStream_t)stream;
        PM_CUDA(cudaMemcpyAsync(p->host, p->rec.d_flag, 4, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaMemcpyAsync(p->host + 1, &p->rec.d_small->status, 4, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaMemcpyAsync(p->host + 2, p->rec.d_nout, 8, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
        const u32 flag = p->host[0], status = p->host[1];
        u64 n = 0;
        memcpy(&n, p->host + 2, 8);
        if (flag & PLAN_MISMATCH) {
            if (n_out) *n_out = 0;
            return PM_EPLAN;
        }
        if (status & ST_INTERNAL) throw Error(PM_ECUDA, "internal consistency check failed");
        if (n_out) *n_out = n;
        return (flag & PLAN_CAPACITY) ? PM_ECAPACITY : PM_OK;
    });
}

// The replay's result into device-accessible page-locked host memory: the
// size is read on the device, so the host waits once.  Nothing is copied
// when the replay did not produce a result (plan flag set) or it exceeds
// the host buffers.
__global__ void k_result_to_host(const u32 *__restrict__ flag, const u64 *__restrict__ nout,
                                 const u64 *__restrict__ keys, const u64 *__restrict__ coefs, u32 words,
                                 u64 *__restrict__ hkeys, u64 *__restrict__ hcoefs, u64 hcap)
{
    const u64 n = *nout;
    if ((flag && *flag) || n > hcap) return;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) hkeys[t] = keys[t];
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < n * words; t += stride) hcoefs[t] = coefs[t];
}

extern "C" int pm_plan_finish_to_host(pm_plan *p, uint64_t *host_keys, void *host_coefs, uint64_t host_cap,
                                      uint64_t *n_out, void *stream)
{
    if (!p || !host_keys || !host_coefs) return PM_EINVAL;
    return guarded([&] {
        cudaStream_t s = (cudaStream_t)stream;
        void *dk = nullptr, *dc = nullptr;
        if (cudaHostGetDevicePointer(&dk, host_keys, 0) != cudaSuccess ||
            cudaHostGetDevicePointer(&dc, host_coefs, 0) != cudaSuccess) {
            cudaGetLastError();
            throw Error(PM_EINVAL, "host buffers are not page-locked and device-accessible");
        }
        const u32 words = p->kind == PM_COEF_M61 ? 1u : (p->kind == PM_COEF_I64_ACC192 ? 3u : 2u);
        int sms = 0, dev = 0;
        PM_CUDA(cudaGetDevice(&dev));
        PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (!p->captured) {
            // the plain call already finished: its size is on the host
            if (p->last_rc != PM_OK) {
                if (n_out) *n_out = p->last_n;
                return p->last_rc;
            }
            if (n_out) *n_out = p->last_n;
            if (p->last_n > host_cap) return PM_ECAPACITY;
            if (p->last_n) {
                PM_CUDA(cudaMemcpyAsync(dk, p->h.keys, p->last_n * 8, cudaMemcpyDeviceToHost, s));
                PM_CUDA(cudaMemcpyAsync(dc, p->h.coefs, p->last_n * 8 * words, cudaMemcpyDeviceToHost, s));
                PM_CUDA(cudaStreamSynchronize(s));
            }
            return PM_OK;
        }
        k_result_to_host<<<sms * 4, 256, 0, s>>>(p->rec.d_flag, p->rec.d_nout, (const u64 *)p->h.keys,
                                                 (const u64 *)p->h.coefs, words, (u64 *)dk, (u64 *)dc, host_cap);
        PM_CUDA(cudaGetLastError());
        PM_CUDA(cudaMemcpyAsync(p->host, p->rec.d_flag, 4, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaMemcpyAsync(p->host + 1, &p->rec.d_small->status, 4, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaMemcpyAsync(p->host + 2, p->rec.d_nout, 8, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
        const u32 flag = p->host[0], status = p->host[1];
        u64 n = 0;
        memcpy(&n, p->host + 2, 8);
        if (flag & PLAN_MISMATCH) {
            if (n_out) *n_out = 0;
            return PM_EPLAN;
        }
        if (status & ST_INTERNAL) throw Error(PM_ECUDA, "internal consistency check failed");
        if (n_out) *n_out = n;
        if (flag & PLAN_CAPACITY) return PM_ECAPACITY;
        return n > host_cap ? PM_ECAPACITY : PM_OK;
    });
}

extern "C" int pm_plan_captured(const pm_plan *p) { return p && p->captured ? 1 : 0; }

extern "C" void pm_plan_destroy(pm_plan *p) { plan_free(p); }

extern "C" const char *pm_strerror(int code)
{
    switch (code) {
    case PM_OK: return "success";
    case PM_EINVAL: return "invalid argument";
    case PM_EEXP_OVERFLOW: return "exponent reaches its field's guard bit";
    case PM_ECOEF_BOUND: return "int128 coefficient bound rule fails";
    case PM_ECAPACITY: return "output capacity too small";
    case PM_ENOMEM: return "device memory allocation failed";
    case PM_ETIMEOUT: return "bounded device wait timed out";
    case PM_ECUDA: return "CUDA runtime error";
    case PM_EPLAN: return "inputs no longer match the plan (re-create it or call pm_polymul)";
    case PM_ECANCELED: return "request cancelled before admission";
    default: return "unknown error";
    }
}

extern "C" int pm_version(void) { return 100; }
