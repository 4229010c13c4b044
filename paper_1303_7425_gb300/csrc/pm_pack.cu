// K-a: monomial packing and operand canonicalisation.
//
// Exponent vectors become 64-bit keys with one guard bit per field (Sec. 7:
// exponents "packed on a 64-bit unsigned integer"; the guard bit is this
// library's overflow rule).  Coefficients are reduced to canonical form, the
// operand is sorted by monomial order and repeated monomials are combined,
// giving the sorted distributed format Sec. 2 assumes for A and B.
#include "pm_pack.cuh"

namespace pm {

// per-variable maximum of the input exponents and the guard-bit check
__global__ void k_maxexp(const u32 *__restrict__ exps, size_t n, u32 nv, Layout L, u32 *__restrict__ maxe,
                         u32 *__restrict__ status)
{
    __shared__ u32 m[PM_MAX_VARS];
    if (threadIdx.x < PM_MAX_VARS) m[threadIdx.x] = 0;
    __syncthreads();
    u32 bad = 0;
    size_t total = n * nv;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        u32 v = (u32)(t % nv);
        u32 e = exps[t];
        if ((u64)e >= (1ull << (L.width[v] - 1))) bad = 1;
        atomicMax(&m[v], e);
    }
    if (bad) atomicOr(status, ST_EXP_OVERFLOW);
    __syncthreads();
    if (threadIdx.x < nv) atomicMax(&maxe[threadIdx.x], m[threadIdx.x]);
}

// key, rank in the (raw) box, canonical coefficient
__global__ void k_pack_terms(const u32 *__restrict__ exps, const void *__restrict__ coefs, size_t n, Layout L,
                             int kind, u64 *__restrict__ key, u64 *__restrict__ rank, u64 *__restrict__ coef)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    u64 k = 0, r = 0;
    for (u32 v = 0; v < L.nv; v++) {
        u64 e = exps[t * L.nv + v];
        k |= e << L.off[v];
        r += e * L.stride[v];
    }
    key[t] = k;
    rank[t] = r;
    u64 c = ((const u64 *)coefs)[t];
    coef[t] = kind == PM_COEF_M61 ? m61_reduce(c) : c;
}

// After the sort: at the head of each run of equal ranks, sum the run's
// coefficients; keep[i] = 1 when i heads a run with a non-zero sum.
__global__ void k_combine_mark(const u64 *__restrict__ rank, const u64 *__restrict__ coef, size_t n, int kind,
                               u64 *__restrict__ val, u64 *__restrict__ keep, u32 *__restrict__ status)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool head = i == 0 || rank[i] != rank[i - 1];
    u64 out = 0;
    bool nz = false;
    if (head) {
        if (kind == PM_COEF_M61) {
            u64 s = coef[i];
            for (size_t j = i + 1; j < n && rank[j] == rank[i]; j++) s = m61_add(s, coef[j]);
            out = s;
            nz = s != 0;
        } else {
            u64 lo = coef[i], hi = (u64)((i64)coef[i] >> 63);
            for (size_t j = i + 1; j < n && rank[j] == rank[i]; j++)
                add128(lo, hi, coef[j], (u64)((i64)coef[j] >> 63));
            // the sum must fit in int64: hi is the sign extension of lo
            if (hi != (u64)((i64)lo >> 63)) atomicOr(status, ST_COEF_BOUND);
            out = lo;
            nz = (lo | hi) != 0;
        }
    }
    val[i] = out;
    keep[i] = (head && nz) ? 1ull : 0ull;
}

__global__ void k_combine_scatter(const u64 *__restrict__ key, const u64 *__restrict__ val,
                                  const u64 *__restrict__ keep, const u64 *__restrict__ pos, size_t n,
                                  u64 *__restrict__ okey, u64 *__restrict__ ocoef)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    okey[pos[i]] = key[i];
    ocoef[pos[i]] = val[i];
}

// per-field maxima of canonical keys, max |coef| (int64 kind), and the
// first and last key; the operand size is read from the device
__global__ void k_operand_stats(const u64 *__restrict__ key, const u64 *__restrict__ coef,
                                const u64 *__restrict__ d_n, Layout L, int kind, u32 *__restrict__ maxe,
                                u64 *__restrict__ maxabs, u64 *__restrict__ first_last)
{
    __shared__ u32 m[PM_MAX_VARS];
    __shared__ u64 ma;
    const size_t n = *d_n;
    if (threadIdx.x < PM_MAX_VARS) m[threadIdx.x] = 0;
    if (threadIdx.x == 0) ma = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && n) {
        first_last[0] = key[0];
        first_last[1] = key[n - 1];
    }
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        u64 k = key[i];
        for (u32 v = 0; v < L.nv; v++) atomicMax(&m[v], key_field(L, k, v));
        if (kind != PM_COEF_M61) {
            i64 c = (i64)coef[i];
            u64 a = c < 0 ? (u64)0 - (u64)c : (u64)c;
            atomicMax(&ma, a);
        }
    }
    __syncthreads();
    if (threadIdx.x < L.nv) atomicMax(&maxe[threadIdx.x], m[threadIdx.x]);
    if (threadIdx.x == 0 && kind != PM_COEF_M61) atomicMax(maxabs, ma);
}

__global__ void k_ranks(const u64 *__restrict__ key, size_t n, Layout L, u64 *__restrict__ rank,
                        u32 *__restrict__ rank32)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const u64 r = key_to_rank(L, key[i]);
        rank[i] = r;
        if (rank32) rank32[i] = (u32)r;
    }
}

__global__ void k_pack_only(const u32 *__restrict__ exps, size_t n, Layout L, u64 *__restrict__ key,
                            u32 *__restrict__ status)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    u64 k = 0;
    for (u32 v = 0; v < L.nv; v++) {
        u64 e = exps[t * L.nv + v];
        if (e >= (1ull << (L.width[v] - 1))) atomicOr(status, ST_EXP_OVERFLOW);
        k |= e << L.off[v];
    }
    key[t] = k;
}

__global__ void k_unpack(const u64 *__restrict__ key, size_t n, Layout L, u32 *__restrict__ exps)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    u64 k = key[t];
    for (u32 v = 0; v < L.nv; v++) exps[t * L.nv + v] = key_field(L, k, v);
}

static unsigned grid_for(size_t n, int threads)
{
    size_t g = (n + threads - 1) / threads;
    return (unsigned)(g ? g : 1);
}

void input_maxima(Ctx &c, const pm_terms_in &in, const Layout &L, u32 *d_maxe, u32 *d_status)
{
    if (in.n == 0) return;
    size_t total = in.n * L.nv;
    unsigned g = grid_for(total, 256);
    if (g > (unsigned)(c.sm_count * 8)) g = c.sm_count * 8;
    k_maxexp<<<g, 256, 0, c.s>>>(in.exps, in.n, L.nv, L, d_maxe, d_status);
    PM_LAUNCHED(c);
}

void canonicalize(Ctx &c, Scratch &S, const pm_terms_in &in, const Layout &raw, u64 raw_box, int kind,
                  Operand &op, u32 *d_status, u64 *d_count)
{
    op.n = 0;
    size_t n = in.n;
    if (n == 0) {
        PM_CUDA(cudaMemsetAsync(d_count, 0, sizeof(u64), c.s));
        op.key = S.get<u64>(1);
        op.coef = S.get<u64>(1);
        op.rank = S.get<u64>(1);
        return;
    }
    u64 *key = S.get<u64>(n), *rank = S.get<u64>(n), *coef = S.get<u64>(n);
    k_pack_terms<<<grid_for(n, 256), 256, 0, c.s>>>(in.exps, in.coefs, n, raw, kind, key, rank, coef);
    PM_LAUNCHED(c);
    radix_sort_pairs(c, S, rank, key, coef, n, bit_length(raw_box - 1));
    u64 *val = S.get<u64>(n), *keep = S.get<u64>(n), *pos = S.get<u64>(n + 1);
    k_combine_mark<<<grid_for(n, 256), 256, 0, c.s>>>(rank, coef, n, kind, val, keep, d_status);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, keep, pos, n);
    op.key = S.get<u64>(n);
    op.coef = S.get<u64>(n);
    op.rank = S.get<u64>(n);
    k_combine_scatter<<<grid_for(n, 256), 256, 0, c.s>>>(key, val, keep, pos, n, op.key, op.coef);
    PM_LAUNCHED(c);
    PM_CUDA(cudaMemcpyAsync(d_count, pos + n, sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
}


// ---------------------------------------------------------------------------
// dense canonicalisation: when an operand's own exponent box is small, each
// term is added into the slot of its rank (repeated monomials combine in the
// slot), then the non-zero slots are compacted in rank order, which is the
// monomial order.  M61: 64-bit sum + 32-bit wrap count (2^64 = 8 mod p);
// I64: 128-bit sum as lo/hi words.
// ---------------------------------------------------------------------------

__global__ void k_dense_scatter(const u32 *__restrict__ exps, const void *__restrict__ coefs, size_t n, Layout L,
                                int kind, u64 *__restrict__ sum, u64 *__restrict__ aux, const u32 *abort)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    // a replayed plan whose inputs left the recorded box stops here: the
    // box below would no longer bound the ranks
    if (t >= n || (abort && *abort)) return;
    u64 r = 0;
    for (u32 v = 0; v < L.nv; v++) r += (u64)exps[t * L.nv + v] * L.stride[v];
    const u64 c = ((const u64 *)coefs)[t];
    if (kind == PM_COEF_M61) {
        const u64 x = m61_reduce(c);
        const u64 old = atomicAdd(&sum[r], x);
        if (old + x < old) atomicAdd((u32 *)aux + r, 1u);
    } else {
        const u64 hi = (u64)((i64)c >> 63);
        const u64 old = atomicAdd(&sum[r], c);
        atomicAdd(&aux[r], hi + (old + c < old ? 1ull : 0ull));
    }
}

__device__ __forceinline__ bool dense_value(const u64 *sum, const u64 *aux, u64 s, int kind, u64 &v, u32 *status)
{
    if (kind == PM_COEF_M61) {
        v = m61_reduce(m61_reduce(sum[s]) + 8ull * ((const u32 *)aux)[s]);
        return v != 0;
    }
    const u64 lo = sum[s], hi = aux[s];
    if (hi != (u64)((i64)lo >> 63) && status) atomicOr(status, ST_COEF_BOUND);  // must fit int64
    v = lo;
    return (lo | hi) != 0;
}

__global__ void k_dense_flags(const u64 *__restrict__ sum, const u64 *__restrict__ aux, u64 box, int kind,
                              u64 *__restrict__ flag, u32 *__restrict__ status)
{
    u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= box) return;
    u64 v;
    flag[s] = dense_value(sum, aux, s, kind, v, status) ? 1ull : 0ull;
}

__global__ void k_dense_emit(const u64 *__restrict__ sum, const u64 *__restrict__ aux, u64 box, int kind,
                             const u64 *__restrict__ flag, const u64 *__restrict__ pos, Layout L,
                             u64 *__restrict__ okey, u64 *__restrict__ ocoef)
{
    u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= box || !flag[s]) return;
    u64 v;
    dense_value(sum, aux, s, kind, v, nullptr);
    okey[pos[s]] = rank_to_key(L, s);
    ocoef[pos[s]] = v;
}

void canonicalize_dense(Ctx &c, Scratch &S, const pm_terms_in &in, const Layout &own, u64 own_box, int kind,
                        Operand &op, u32 *d_status, u64 *d_count, const u32 *abort)
{
    op.n = 0;
    const size_t n = in.n;
    u64 *sum = S.get<u64>(own_box), *aux = S.get<u64>(own_box);
    PM_CUDA(cudaMemsetAsync(sum, 0, own_box * 8, c.s));
    PM_CUDA(cudaMemsetAsync(aux, 0, own_box * 8, c.s));
    k_dense_scatter<<<grid_for(n, 256), 256, 0, c.s>>>(in.exps, in.coefs, n, own, kind, sum, aux, abort);
    PM_LAUNCHED(c);
    u64 *flag = S.get<u64>(own_box), *pos = S.get<u64>(own_box + 1);
    k_dense_flags<<<grid_for(own_box, 256), 256, 0, c.s>>>(sum, aux, own_box, kind, flag, d_status);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, flag, pos, own_box);
    const size_t cap = n < own_box ? n : own_box;
    op.key = S.get<u64>(cap);
    op.coef = S.get<u64>(cap);
    op.rank = S.get<u64>(cap);
    k_dense_emit<<<grid_for(own_box, 256), 256, 0, c.s>>>(sum, aux, own_box, kind, flag, pos, own, op.key,
                                                          op.coef);
    PM_LAUNCHED(c);
    PM_CUDA(cudaMemcpyAsync(d_count, pos + own_box, sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
}

void operand_stats(Ctx &c, const Operand &op, u64 n_max, const u64 *d_n, const Layout &L, int kind, u32 *d_maxe,
                   u64 *d_maxabs, u64 *d_first_last)
{
    if (n_max == 0) return;
    unsigned g = grid_for(n_max, 256);
    if (g > (unsigned)(c.sm_count * 4)) g = c.sm_count * 4;
    k_operand_stats<<<g, 256, 0, c.s>>>(op.key, op.coef, d_n, L, kind, d_maxe, d_maxabs, d_first_last);
    PM_LAUNCHED(c);
}

void operand_ranks(Ctx &c, Operand &op, const Layout &L, u32 *rank32)
{
    if (op.n == 0) return;
    k_ranks<<<grid_for(op.n, 256), 256, 0, c.s>>>(op.key, op.n, L, op.rank, rank32);
    PM_LAUNCHED(c);
}

void pack_keys(Ctx &c, const u32 *exps, size_t n, const Layout &L, u64 *keys, u32 *d_status)
{
    if (n == 0) return;
    k_pack_only<<<grid_for(n, 256), 256, 0, c.s>>>(exps, n, L, keys, d_status);
    PM_LAUNCHED(c);
}

void unpack_keys(Ctx &c, const u64 *keys, size_t n, const Layout &L, u32 *exps)
{
    if (n == 0) return;
    k_unpack<<<grid_for(n, 256), 256, 0, c.s>>>(keys, n, L, exps);
    PM_LAUNCHED(c);
}

}  // namespace pm
