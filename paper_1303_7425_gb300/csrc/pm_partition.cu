// K-b: splitting the output exponent space into disjoint ranges.
//
// The pp-matrix gamma_{i,j} = alpha_i + beta_j (Sec. 2, Fig. 1) is strictly
// increasing along rows and columns, so the number of term products below a
// bound x is sum_i #{j : beta_j < x - alpha_i}, one lower-bound search per
// row.  Counting at every splitter gives the operation counts O_k of
// Alg. 2 (Sec. 3); ranges whose count is above the target are split further
// (by key value) until the target holds or the range is a single monomial.
// The first splitter set is either the almost regular grid of Sec. 5 or a
// uniform split of the rank box (direct-addressed strategy).
#include "pm_partition.cuh"

namespace pm {

constexpr int KB_THREADS = 256;

// cnt[k] = #{(i, j) : A_i + B_j < S_k}
__global__ void __launch_bounds__(KB_THREADS) k_count_below(const u64 *__restrict__ A, u32 na,
                                                            const u64 *__restrict__ B, u32 nb,
                                                            const u64 *__restrict__ Sp, u32 ns,
                                                            u64 *__restrict__ cnt)
{
    __shared__ u64 ws[32];
    __shared__ u32 rows[2];
    const u64 blast = B[nb - 1];
    for (u32 k = blockIdx.x; k < ns; k += gridDim.x) {
        const u64 x = Sp[k];
        if (threadIdx.x == 0) {
            rows[0] = x > blast ? lower_bound_u64(A, na, x - blast) : 0;  // full rows
            rows[1] = lower_bound_u64(A, na, x);                           // rows with any column
        }
        __syncthreads();
        const u32 ifull = rows[0], iz = rows[1];
        u64 s = 0;
        for (u32 i = ifull + threadIdx.x; i < iz; i += blockDim.x) s += lower_bound_u64(B, nb, x - A[i]);
        u64 total;
        block_exclusive_scan(s, total, ws);
        if (threadIdx.x == 0) cnt[k] = total + (u64)ifull * nb;
        __syncthreads();
    }
}

// S[m] = min(lo + m * step, end), m = 0..M (S[M] = end)
__global__ void k_uniform_splitters(u64 lo, u64 end, u64 step, u32 M, u64 *__restrict__ Sp)
{
    u32 m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > M) return;
    u64 v = lo + (u64)m * step;
    Sp[m] = (m == M || v > end) ? end : v;
}

// the Sec. 5 grid's points (grid_point)
__global__ void k_grid(const u64 *__restrict__ A, u32 na, const u64 *__restrict__ B, u32 nb, GridShape g,
                       u64 *__restrict__ out)
{
    const u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.total) return;
    u64 i, j;
    grid_point(g, na, nb, p, i, j);
    out[p] = A[i] + B[j];
}

__global__ void k_set_u64(u64 *p, u64 v) { *p = v; }

__global__ void k_clamp(u64 *__restrict__ v, size_t n, u64 lo, u64 hi)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = v[i] < lo ? lo : (v[i] > hi ? hi : v[i]);
}

__global__ void k_unique_mark(const u64 *__restrict__ v, size_t n, u64 *__restrict__ keep)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = (i == 0 || v[i] != v[i - 1]) ? 1ull : 0ull;
}

__global__ void k_select(const u64 *__restrict__ v, const u64 *__restrict__ keep, const u64 *__restrict__ pos,
                         size_t n, u64 *__restrict__ out)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && keep[i]) out[pos[i]] = v[i];
}

// pieces per range: 1 if O_k <= target (or the range is one monomial)
__global__ void k_refine_plan(const u64 *__restrict__ Sp, const u64 *__restrict__ cnt, u32 nr, u64 target,
                              u64 max_q, u64 *__restrict__ q)
{
    u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    u64 O = cnt[k + 1] - cnt[k];
    u64 span = Sp[k + 1] - Sp[k];
    u64 pieces = 1;
    if (O > target && span > 1) {
        pieces = (O + target - 1) / target;
        if (pieces < 2) pieces = 2;
        if (pieces > max_q) pieces = max_q;
        if (pieces > span) pieces = span;
    }
    q[k] = pieces;
}

__global__ void k_refine_emit(const u64 *__restrict__ Sp, u32 nr, const u64 *__restrict__ q,
                              const u64 *__restrict__ pos, u64 *__restrict__ Snew)
{
    u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    u64 lo = Sp[k], span = Sp[k + 1] - lo, pieces = q[k], base = pos[k];
    for (u64 m = 0; m < pieces; m++)
        Snew[base + m] = lo + (u64)(((unsigned __int128)span * m) / pieces);
    if (k == nr - 1) Snew[pos[nr]] = Sp[nr];
}

// final range list: ranges with O_k > 0, with their bounds and output bounds
__global__ void k_ranges_mark(const u64 *__restrict__ cnt, u32 nr, u64 *__restrict__ keep)
{
    u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nr) keep[k] = cnt[k + 1] > cnt[k] ? 1ull : 0ull;
}

__global__ void k_ranges_emit(const u64 *__restrict__ Sp, const u64 *__restrict__ cnt, u32 nr,
                              const u64 *__restrict__ keep, const u64 *__restrict__ pos, u64 *__restrict__ rlo,
                              u64 *__restrict__ rhi, u64 *__restrict__ rO, u64 *__restrict__ rbound)
{
    u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr || !keep[k]) return;
    u64 o = cnt[k + 1] - cnt[k], span = Sp[k + 1] - Sp[k];
    u64 d = pos[k];
    rlo[d] = Sp[k];
    rhi[d] = Sp[k + 1];
    rO[d] = o;
    rbound[d] = o < span ? o : span;
}

static unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t ? (n + t - 1) / t : 1); }

void grid_sample(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const GridShape &g, u64 *out)
{
    k_grid<<<blocks_for(g.total, 256), 256, 0, c.s>>>(A, na, B, nb, g, out);
    PM_LAUNCHED(c);
}

void split_cumulative(const u64 *cum, u32 ns, u32 nshards, u32 *cut)
{
    const u64 total = ns ? cum[ns - 1] : 0;
    cut[0] = 0;
    u32 k = 0;
    for (u32 m = 1; m < nshards; m++) {
        const unsigned __int128 want = (unsigned __int128)total * m;  // cum[k] * nshards >= total * m
        while (k + 1 < ns && (unsigned __int128)cum[k] * nshards < want) k++;
        cut[m] = k;
    }
    cut[nshards] = ns ? ns - 1 : 0;
}

void count_below(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const u64 *Sp, u32 ns, u64 *cnt);

static void count_at(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const u64 *Sp, u32 ns, u64 *cnt)
{
    count_below(c, A, na, B, nb, Sp, ns, cnt);
}

void count_below(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const u64 *Sp, u32 ns, u64 *cnt)
{
    unsigned g = ns < (u32)(c.sm_count * 16) ? ns : (unsigned)(c.sm_count * 16);
    k_count_below<<<g, KB_THREADS, 0, c.s>>>(A, na, B, nb, Sp, ns, cnt);
    PM_LAUNCHED(c);
}

static u64 read_u64(Ctx &c, const u64 *d)
{
    u64 h = 0;
    PM_CUDA(cudaMemcpyAsync(&h, d, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    c.sync();
    return h;
}

u64 *grid_splitters(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u32 l, u64 end, u32 *ns,
                    u64 clamp_lo, u64 clamp_hi)
{
    const GridShape g = grid_shape(na, nb, l);
    u64 total = g.total;
    u64 *cand = S.get<u64>(total + 1);
    grid_sample(c, A, na, B, nb, g, cand);
    k_set_u64<<<1, 1, 0, c.s>>>(cand + total, end);  // gamma_end
    PM_LAUNCHED(c);
    total += 1;
    radix_sort_pairs(c, S, cand, nullptr, nullptr, total, bit_length(end));
    if (clamp_lo != 0 || clamp_hi != ~0ull) {  // monotone: the order holds
        k_clamp<<<blocks_for(total, 256), 256, 0, c.s>>>(cand, total, clamp_lo, clamp_hi);
        PM_LAUNCHED(c);
    }
    u64 *keep = S.get<u64>(total), *pos = S.get<u64>(total + 1);
    k_unique_mark<<<blocks_for(total, 256), 256, 0, c.s>>>(cand, total, keep);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, keep, pos, total);
    u64 *Sp = S.get<u64>(total);
    k_select<<<blocks_for(total, 256), 256, 0, c.s>>>(cand, keep, pos, total, Sp);
    PM_LAUNCHED(c);
    *ns = (u32)read_u64(c, pos + total);
    return Sp;
}

Ranges partition(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, const PartitionPlan &plan)
{
    // host copies of the key extremes (four words)
    u64 ext[4];
    PM_CUDA(cudaMemcpyAsync(&ext[0], A, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    PM_CUDA(cudaMemcpyAsync(&ext[1], A + na - 1, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    PM_CUDA(cudaMemcpyAsync(&ext[2], B, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    PM_CUDA(cudaMemcpyAsync(&ext[3], B + nb - 1, sizeof(u64), cudaMemcpyDeviceToHost, c.s));
    c.sync();
    u64 lo = ext[0] + ext[2];
    u64 end = ext[1] + ext[3] + 1;  // gamma_end: one past the largest product key
    // a slice of the output key space: the caller checked it is not empty
    if (plan.key_lo > lo) lo = plan.key_lo;
    if (plan.key_hi < end) end = plan.key_hi;
    if (lo >= end) throw Error(PM_ECUDA, "empty key slice reached the partition");

    u64 *Sp = nullptr;
    u32 ns = 0;  // number of boundaries (ranges + 1)
    if (plan.uniform_step) {
        u64 M = (end - lo + plan.uniform_step - 1) / plan.uniform_step;
        if (M > plan.max_ranges) throw Error(PM_ENOMEM, "too many ranges");
        ns = (u32)M + 1;
        Sp = S.get<u64>(ns);
        k_uniform_splitters<<<blocks_for(ns, 256), 256, 0, c.s>>>(lo, end, plan.uniform_step, (u32)M, Sp);
        PM_LAUNCHED(c);
    } else {
        // Sec. 5 grid with parameter l, steps clamped to >= 1
        Sp = grid_splitters(c, S, A, na, B, nb, plan.grid_l ? plan.grid_l : 1, ext[1] + ext[3] + 1, &ns, lo, end);
    }

    // count, then refine ranges above the target
    u64 *cnt = S.get<u64>(ns);
    count_at(c, A, na, B, nb, Sp, ns, cnt);
    u32 rounds = 0;
    for (; rounds < plan.max_rounds; rounds++) {
        u32 nr = ns - 1;
        u64 *q = S.get<u64>(nr), *pos = S.get<u64>(nr + 1);
        k_refine_plan<<<blocks_for(nr, 256), 256, 0, c.s>>>(Sp, cnt, nr, plan.target, plan.max_split, q);
        PM_LAUNCHED(c);
        scan_exclusive_u64(c, S, q, pos, nr);
        u64 nr_new = read_u64(c, pos + nr);
        if (nr_new == nr) break;
        if (nr_new + 1 > plan.max_ranges) {
            if (plan.hard_target) throw Error(PM_ENOMEM, "partition exceeds the range limit");
            break;
        }
        u64 *Snew = S.get<u64>(nr_new + 1);
        k_refine_emit<<<blocks_for(nr, 256), 256, 0, c.s>>>(Sp, nr, q, pos, Snew);
        PM_LAUNCHED(c);
        Sp = Snew;
        ns = (u32)nr_new + 1;
        cnt = S.get<u64>(ns);
        count_at(c, A, na, B, nb, Sp, ns, cnt);
    }

    // keep the non-empty ranges
    Ranges R;
    R.rounds = rounds;
    u32 nr = ns - 1;
    u64 *keep = S.get<u64>(nr), *pos = S.get<u64>(nr + 1);
    k_ranges_mark<<<blocks_for(nr, 256), 256, 0, c.s>>>(cnt, nr, keep);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, keep, pos, nr);
    u64 nk = read_u64(c, pos + nr);
    R.n = (u32)nk;
    R.lo = S.get<u64>(nk + 1);
    R.hi = S.get<u64>(nk + 1);
    R.O = S.get<u64>(nk + 1);
    u64 *bound = S.get<u64>(nk + 1);
    R.boff = S.get<u64>(nk + 1);
    k_ranges_emit<<<blocks_for(nr, 256), 256, 0, c.s>>>(Sp, cnt, nr, keep, pos, R.lo, R.hi, R.O, bound);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, bound, R.boff, nk);
    R.out_bound = read_u64(c, R.boff + nk);
    return R;
}

}  // namespace pm
