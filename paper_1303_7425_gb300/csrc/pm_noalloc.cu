// pm_polymul_noalloc: the product for callers that cannot allocate device
// memory (include/polymul.h).
//
// Some callers cannot call cudaMalloc or any allocator: code that runs
// where allocation is forbidden or would synchronise the device (a
// real-time or latency-critical thread, an allocator callback, a plugin
// whose host application owns every device allocation).  This entry point
// serves small products for them.  It runs one kernel, a single-CTA variant
// of the sort-and-reduce range kernel that treats the whole product as one
// range; all of its scratch lives in the file-scope static device array
// below, which every GPU that loads the library keeps until the process
// exits.  The caller passes inputs and outputs as for pm_polymul.
//
// Every call shares that array and it keeps the last call's contents; the
// kernel clears what must start at zero itself.  Calls whose executions
// overlap on the GPU (on different streams, or from different host
// threads) race on the array: callers must serialise them.
#include <cstring>
#include <mutex>

#include "pm_common.cuh"

namespace pm {

constexpr u32 NA_MAX_TERMS = PM_NOALLOC_MAX_TERMS;
constexpr u32 NA_MAX_PRODUCTS = PM_NOALLOC_MAX_PRODUCTS;
constexpr int NT = 1024;  // threads of the single CTA

// scratch layout (bytes), all offsets multiples of 256
struct NaLayout {
    static constexpr size_t head = 0;                                    // status words
    static constexpr size_t opnd = 256;                                  // per operand below
    static constexpr size_t opnd_bytes = (size_t)NA_MAX_TERMS * (8 + 8 + 8 + 4 + 4 + 8 + 8);
    static constexpr size_t prod = opnd + 2 * opnd_bytes;
    static constexpr size_t prod_bytes = (size_t)NA_MAX_PRODUCTS * (8 + 8 + 4 + 4 + 8 + 8);
    static constexpr size_t total = prod + prod_bytes;
};
static_assert(NaLayout::total <= PM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the static array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PM_NOALLOC_SCRATCH_BYTES];

struct NaHead {
    u32 status;
    u32 n_f, n_g;
    u32 pad;
    u64 n_out;
};

struct NaOperand {  // views into the scratch
    u64 *k, *k2;     // keys and sort buffer
    u64 *c;          // canonical coefficient of the raw term
    u32 *ix, *ix2;   // sort payload
    u64 *ck, *cc;    // canonical operand: keys, coefficients
};

__device__ __forceinline__ NaOperand na_operand(unsigned char *base)
{
    NaOperand o;
    o.k = (u64 *)base;
    o.k2 = o.k + NA_MAX_TERMS;
    o.c = o.k2 + NA_MAX_TERMS;
    o.ck = o.c + NA_MAX_TERMS;
    o.cc = o.ck + NA_MAX_TERMS;
    o.ix = (u32 *)(o.cc + NA_MAX_TERMS);
    o.ix2 = o.ix + NA_MAX_TERMS;
    return o;
}

struct NaShared {
    u32 hist[256];
    u32 base[256];
    u32 wcnt[NT / 32][256];
    u64 ws[32];
    u32 maxe[2][PM_MAX_VARS];
    u64 maxabs[2];
    u64 orv, andv;
};

// Stable LSD radix sort of n (key, index) pairs held in global scratch, by
// one CTA: per 8-bit digit a histogram, then a scatter in index order, tile
// by tile, with ranks from warp match masks and per-warp digit counts.
__device__ void na_sort(u64 *&k, u32 *&ix, u64 *&k2, u32 *&ix2, u32 n, NaShared &sh)
{
    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        sh.orv = 0;
        sh.andv = ~0ull;
    }
    __syncthreads();
    u64 o = 0, a = ~0ull;
    for (u32 i = tid; i < n; i += NT) {
        o |= k[i];
        a &= k[i];
    }
    atomicOr(&sh.orv, o);
    atomicAnd(&sh.andv, a);
    __syncthreads();
    const u64 vary = sh.orv ^ sh.andv;
    int hi = 64;
    while (hi > 0 && !((vary >> (hi - 1)) & 1)) hi--;
    __syncthreads();
    for (int shift = 0; shift < hi; shift += 8) {
        if (tid < 256) sh.hist[tid] = 0;
        __syncthreads();
        for (u32 i = tid; i < n; i += NT) atomicAdd(&sh.hist[(k[i] >> shift) & 255u], 1u);
        __syncthreads();
        u64 tot;
        const u64 ex = block_exclusive_scan(tid < 256 ? sh.hist[tid] : 0, tot, sh.ws);
        if (tid < 256) sh.base[tid] = (u32)ex;
        __syncthreads();
        for (u32 t0 = 0; t0 < n; t0 += NT) {
            for (u32 x = tid; x < (NT / 32) * 256; x += NT) (&sh.wcnt[0][0])[x] = 0;
            __syncthreads();
            const u32 i = t0 + tid;
            const bool valid = i < n;
            const u32 d = valid ? (u32)((k[i] >> shift) & 255u) : 256u;
            const u32 peers = __match_any_sync(0xffffffffu, d);
            const u32 lt = __popc(peers & ((1u << lane) - 1u));
            if (valid && lt == 0) sh.wcnt[w][d] = __popc(peers);
            __syncthreads();
            if (tid < 256) {  // exclusive prefix over warps, and the tile's total
                u32 run = 0;
                for (int ww = 0; ww < NT / 32; ww++) {
                    const u32 c = sh.wcnt[ww][tid];
                    sh.wcnt[ww][tid] = run;
                    run += c;
                }
                sh.hist[tid] = run;
            }
            __syncthreads();
            if (valid) {
                const u32 pos = sh.base[d] + sh.wcnt[w][d] + lt;
                k2[pos] = k[i];
                ix2[pos] = ix[i];
            }
            __syncthreads();
            if (tid < 256) sh.base[tid] += sh.hist[tid];
            __syncthreads();
        }
        u64 *tk = k;
        k = k2;
        k2 = tk;
        u32 *ti = ix;
        ix = ix2;
        ix2 = ti;
    }
}

// pack an operand's terms: key, canonical coefficient, identity index
__device__ void na_pack(const u32 *exps, const u64 *coefs, u32 n, const Layout &L, int kind, NaOperand &o, u32 *st)
{
    for (u32 t = threadIdx.x; t < n; t += NT) {
        u64 key = 0;
        for (u32 v = 0; v < L.nv; v++) {
            const u64 e = exps[(size_t)t * L.nv + v];
            if (e >= (1ull << (L.width[v] - 1))) atomicOr(st, ST_EXP_OVERFLOW);
            key |= e << L.off[v];
        }
        o.k[t] = key;
        o.c[t] = kind == PM_COEF_M61 ? m61_reduce(coefs[t]) : coefs[t];
        o.ix[t] = t;
    }
}

// combine equal keys of a sorted operand and drop zero sums; returns the
// canonical size (all threads)
__device__ u32 na_combine(const u64 *k, const u32 *ix, const u64 *c, u32 n, int kind, u64 *ck, u64 *cc, u32 *st,
                          NaShared &sh)
{
    u32 run = 0;
    for (u32 t0 = 0; t0 < n; t0 += NT) {
        const u32 i = t0 + threadIdx.x;
        u64 v = 0;
        bool nz = false;
        if (i < n && (i == 0 || k[i] != k[i - 1])) {
            if (kind == PM_COEF_M61) {
                for (u32 j = i; j < n && k[j] == k[i]; j++) v = m61_add(v, c[ix[j]]);
                nz = v != 0;
            } else {
                u64 lo = 0, hi = 0;
                for (u32 j = i; j < n && k[j] == k[i]; j++) add128(lo, hi, c[ix[j]], (u64)((i64)c[ix[j]] >> 63));
                if (hi != (u64)((i64)lo >> 63)) atomicOr(st, ST_COEF_BOUND);
                v = lo;
                nz = (lo | hi) != 0;
            }
        }
        u64 cnt;
        const u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, sh.ws);
        if (nz) {
            ck[run + pos] = k[i];
            cc[run + pos] = v;
        }
        run += (u32)cnt;
    }
    __syncthreads();
    return run;
}

__global__ void __launch_bounds__(NT, 1) k_small_product(unsigned char *scr, Layout L, int kind,
                                                         const u32 *fe, const u64 *fc, u32 nf, const u32 *ge,
                                                         const u64 *gc, u32 ng, u64 *hkey, u64 *hcoef, u64 cap)
{
    __shared__ NaShared sh;
    NaHead *head = (NaHead *)(scr + NaLayout::head);
    u32 *st = &head->status;
    const u32 tid = threadIdx.x;
    if (tid == 0) {  // the scratch keeps the previous call's contents
        head->status = 0;
        head->n_f = head->n_g = 0;
        head->n_out = 0;
    }
    if (tid < 2 * PM_MAX_VARS) (&sh.maxe[0][0])[tid] = 0;
    if (tid < 2) sh.maxabs[tid] = 0;
    __syncthreads();
    NaOperand F = na_operand(scr + NaLayout::opnd), G = na_operand(scr + NaLayout::opnd + NaLayout::opnd_bytes);

    // canonical operands (the sorted distributed format of Sec. 2)
    na_pack(fe, fc, nf, L, kind, F, st);
    na_pack(ge, gc, ng, L, kind, G, st);
    __syncthreads();
    if (*st) return;
    na_sort(F.k, F.ix, F.k2, F.ix2, nf, sh);
    na_sort(G.k, G.ix, G.k2, G.ix2, ng, sh);
    const u32 cf = na_combine(F.k, F.ix, F.c, nf, kind, F.ck, F.cc, st, sh);
    const u32 cg = na_combine(G.k, G.ix, G.c, ng, kind, G.ck, G.cc, st, sh);
    if (tid == 0) {
        head->n_f = cf;
        head->n_g = cg;
    }
    __syncthreads();
    if (*st || cf == 0 || cg == 0) return;

    // the product's largest exponents and coefficient bound
    for (u32 t = tid; t < cf + cg; t += NT) {
        const int q = t < cf ? 0 : 1;
        const u64 key = q ? G.ck[t - cf] : F.ck[t];
        const u64 c = q ? G.cc[t - cf] : F.cc[t];
        for (u32 v = 0; v < L.nv; v++) atomicMax(&sh.maxe[q][v], key_field(L, key, v));
        if (kind != PM_COEF_M61) atomicMax(&sh.maxabs[q], (i64)c < 0 ? (u64)0 - c : c);
    }
    __syncthreads();
    if (tid == 0) {
        for (u32 v = 0; v < L.nv; v++)
            if ((u64)sh.maxe[0][v] + sh.maxe[1][v] >= (1ull << (L.width[v] - 1))) atomicOr(st, ST_EXP_OVERFLOW);
        if (kind != PM_COEF_M61) {
            const unsigned __int128 m = (unsigned __int128)sh.maxabs[0] * sh.maxabs[1];
            const unsigned __int128 lim = ((((unsigned __int128)1) << 127) - 1) / (cf < cg ? cf : cg);
            if (m > lim) atomicOr(st, ST_COEF_BOUND);
        }
    }
    __syncthreads();
    if (*st) return;
    const u32 np = cf * cg;
    if (np > NA_MAX_PRODUCTS) {  // the host checks raw sizes; canonical ones are smaller
        if (tid == 0) atomicOr(st, ST_CAPACITY | ST_INTERNAL);
        return;
    }

    // every pairwise term product (Sec. 2), then one sort + segmented reduce
    unsigned char *pb = scr + NaLayout::prod;
    u64 *pk = (u64 *)pb, *pk2 = pk + NA_MAX_PRODUCTS, *pc = pk2 + NA_MAX_PRODUCTS;  // pc: lo then hi words
    u32 *pi = (u32 *)(pc + 2 * (size_t)NA_MAX_PRODUCTS), *pi2 = pi + NA_MAX_PRODUCTS;
    for (u32 p = tid; p < np; p += NT) {
        const u32 i = p / cg, j = p - i * cg;
        pk[p] = F.ck[i] + G.ck[j];
        pi[p] = p;
        if (kind == PM_COEF_M61) {
            pc[p] = m61_reduce(m61_mul_lazy(F.cc[i], G.cc[j]));
        } else {
            u64 lo, hi;
            mul_i64_wide((i64)F.cc[i], (i64)G.cc[j], lo, hi);
            pc[p] = lo;
            pc[NA_MAX_PRODUCTS + p] = hi;
        }
    }
    __syncthreads();
    na_sort(pk, pi, pk2, pi2, np, sh);
    u64 run = 0;
    for (u32 t0 = 0; t0 < np; t0 += NT) {
        const u32 i = t0 + tid;
        u64 v0 = 0, v1 = 0;
        bool nz = false;
        if (i < np && (i == 0 || pk[i] != pk[i - 1])) {
            for (u32 j = i; j < np && pk[j] == pk[i]; j++) {
                if (kind == PM_COEF_M61) v0 = m61_add(v0, pc[pi[j]]);
                else add128(v0, v1, pc[pi[j]], pc[NA_MAX_PRODUCTS + pi[j]]);
            }
            nz = (v0 | v1) != 0;
        }
        u64 cnt;
        const u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, sh.ws);
        const u64 d = run + pos;
        if (nz && d < cap) {
            hkey[d] = pk[i];
            if (kind == PM_COEF_M61) {
                hcoef[d] = v0;
            } else {
                hcoef[2 * d] = v0;
                hcoef[2 * d + 1] = v1;
            }
        }
        run += cnt;
    }
    if (tid == 0) {
        head->n_out = run;
        if (run > cap) atomicOr(st, ST_CAPACITY);
    }
}

// per-device address of the static scratch, looked up once per device
static std::mutex g_na_mu;
static unsigned char *g_na_ptr[64];

static unsigned char *noalloc_scratch()
{
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(PM_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            throw Error(PM_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_na_ptr[dev] = (unsigned char *)p;
    }
    return g_na_ptr[dev];
}

static int polymul_noalloc_impl(const pm_packing *pk, int kind, const pm_terms_in *f, const pm_terms_in *g,
                                pm_terms_out *h, cudaStream_t s)
{
    if (!pk || pk->nvars < 1 || pk->nvars > PM_MAX_VARS) throw Error(PM_EINVAL, "bad nvars");
    if (kind != PM_COEF_M61 && kind != PM_COEF_I64_ACC128) throw Error(PM_EINVAL, "bad coefficient kind");
    if (!f || !g || !h) throw Error(PM_EINVAL, "null argument");
    if ((f->n && (!f->exps || !f->coefs)) || (g->n && (!g->exps || !g->coefs))) throw Error(PM_EINVAL, "null arrays");
    if (h->cap && (!h->keys || !h->coefs)) throw Error(PM_EINVAL, "null output arrays");
    if (f->n > NA_MAX_TERMS || g->n > NA_MAX_TERMS || f->n * g->n > NA_MAX_PRODUCTS)
        throw Error(PM_EINVAL, "operands exceed the static scratch (PM_NOALLOC_MAX_TERMS / _PRODUCTS)");
    Layout L;
    memset(&L, 0, sizeof(L));
    L.nv = pk->nvars;
    u32 sum = 0;
    for (int v = (int)pk->nvars - 1; v >= 0; v--) {
        const u32 wv = pk->field_bits[v];
        if (wv < 1 || wv > 32) throw Error(PM_EINVAL, "bad field width");
        L.off[v] = sum;
        L.width[v] = wv;
        sum += wv;
    }
    if (sum > 64) throw Error(PM_EINVAL, "fields exceed 64 bits");
    h->n = 0;
    if (f->n == 0 || g->n == 0) return PM_OK;
    unsigned char *scr = noalloc_scratch();
    k_small_product<<<1, NT, 0, s>>>(scr, L, kind, f->exps, (const u64 *)f->coefs, (u32)f->n, g->exps,
                                     (const u64 *)g->coefs, (u32)g->n, (u64 *)h->keys, (u64 *)h->coefs, h->cap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(PM_ECUDA, cudaGetErrorString(e));
    NaHead hd;
    PM_CUDA(cudaMemcpyAsync(&hd, scr + NaLayout::head, sizeof(hd), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (hd.status & ST_INTERNAL) throw Error(PM_ECUDA, "internal consistency check failed");
    if (hd.status & ST_EXP_OVERFLOW) return PM_EEXP_OVERFLOW;
    if (hd.status & ST_COEF_BOUND) return PM_ECOEF_BOUND;
    if (hd.status & ST_CAPACITY) {
        h->n = hd.n_out;
        return PM_ECAPACITY;
    }
    h->n = hd.n_out;
    return PM_OK;
}

}  // namespace pm

extern "C" int pm_polymul_noalloc(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                                  pm_terms_out *h, void *stream)
{
    int rc;
    try {
        rc = pm::polymul_noalloc_impl(pk, coef_kind, f, g, h, (cudaStream_t)stream);
    } catch (const pm::Error &e) {
        rc = e.code;
    } catch (...) {
        rc = PM_ECUDA;
    }
    if (rc != PM_OK && rc != PM_ECAPACITY && h) h->n = 0;
    return rc;
}
