/* Oracle for the sparse multivariate polynomial product -- TEST
 * INFRASTRUCTURE ONLY (see oracle.h).  Plain, slow, obviously correct C.
 *
 * Coefficient arithmetic is written as its definition: x mod p with the C
 * remainder operator on 128-bit integers, p = 2^61 - 1; the int64 kind adds
 * exact 128-bit products.  No reduction tricks, no packing in oracle_mul.
 */
#define _GNU_SOURCE 1
#include "oracle.h"

#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0 /* 0 in every real build; see tests/test_oracle_mutations.py */
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

static const uint64_t P61 = 0x1FFFFFFFFFFFFFFFULL; /* 2^61 - 1 */

/* ------------------------------------------------------------------ */
/* coefficient arithmetic (definitions)                                */
/* ------------------------------------------------------------------ */

static uint64_t m61_of_u64(uint64_t x) { return x % P61; }
static uint64_t m61_add(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a + b) % P61); }
static uint64_t m61_mul(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) % P61); }

static uint64_t m61_of_i128(i128 x)
{
    i128 r = x % (i128)P61;
    if (r < 0) r += (i128)P61;
    return (uint64_t)r;
}

/* A coefficient in either ring is held as an i128: the residue in [0, p)
 * for kind 0, the exact integer for kind 1. */
static i128 coef_in(int kind, const void *coefs, uint64_t t)
{
    if (kind == OR_KIND_M61) return (i128)m61_of_u64(((const uint64_t *)coefs)[t]);
    return (i128)((const int64_t *)coefs)[t];
}

static i128 coef_add(int kind, i128 a, i128 b)
{
    if (kind == OR_KIND_M61) return (i128)m61_add((uint64_t)a, (uint64_t)b);
    return a + b;
}

static i128 coef_mul(int kind, i128 a, i128 b)
{
    if (kind == OR_KIND_M61) return (i128)m61_mul((uint64_t)a, (uint64_t)b);
    return a * b; /* |a|, |b| <= 2^63: the product fits in 127 bits */
}

static void coef_out(int kind, i128 c, void *out, uint64_t t)
{
    if (kind == OR_KIND_M61) {
        ((uint64_t *)out)[t] = (uint64_t)c;
    } else {
        u128 u = (u128)c;
        ((uint64_t *)out)[2 * t] = (uint64_t)u;
        ((uint64_t *)out)[2 * t + 1] = (uint64_t)(u >> 64);
    }
}

/* ------------------------------------------------------------------ */
/* hash map: exponent vector -> coefficient                            */
/* ------------------------------------------------------------------ */

typedef struct {
    uint32_t nv;
    uint64_t cap, used;
    uint32_t *keys;
    uint8_t *full;
    i128 *val;
} vmap;

static uint64_t hash_vec(const uint32_t *e, uint32_t nv)
{
    uint64_t h = 1469598103934665603ULL; /* FNV-1a offset basis */
    for (uint32_t v = 0; v < nv; v++) {
        h ^= e[v];
        h *= 1099511628211ULL;
    }
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdULL;
    h ^= h >> 33;
    return h;
}

static int vmap_alloc(vmap *m, uint32_t nv, uint64_t cap)
{
    m->nv = nv;
    m->cap = cap;
    m->used = 0;
    m->keys = (uint32_t *)malloc(cap * nv * sizeof(uint32_t));
    m->full = (uint8_t *)calloc(cap, 1);
    m->val = (i128 *)malloc(cap * sizeof(i128));
    if (!m->keys || !m->full || !m->val) {
        free(m->keys); free(m->full); free(m->val);
        return OR_ENOMEM;
    }
    return OR_OK;
}

static void vmap_free(vmap *m)
{
    free(m->keys); free(m->full); free(m->val);
    m->keys = NULL; m->full = NULL; m->val = NULL;
}

static int vmap_init(vmap *m, uint32_t nv, uint64_t expect)
{
    uint64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    return vmap_alloc(m, nv, cap);
}

static i128 *vmap_find(const vmap *m, const uint32_t *e)
{
    uint64_t h = hash_vec(e, m->nv) & (m->cap - 1);
    while (m->full[h]) {
        if (memcmp(m->keys + h * m->nv, e, m->nv * sizeof(uint32_t)) == 0) return &m->val[h];
        h = (h + 1) & (m->cap - 1);
    }
    return NULL;
}

static int vmap_grow(vmap *m);

/* Find the slot of e, inserting it with value 0 when absent. */
static i128 *vmap_slot(vmap *m, const uint32_t *e)
{
    if (2 * (m->used + 1) > m->cap && vmap_grow(m) != OR_OK) return NULL;
    uint64_t h = hash_vec(e, m->nv) & (m->cap - 1);
    while (m->full[h]) {
        if (memcmp(m->keys + h * m->nv, e, m->nv * sizeof(uint32_t)) == 0) return &m->val[h];
        h = (h + 1) & (m->cap - 1);
    }
    memcpy(m->keys + h * m->nv, e, m->nv * sizeof(uint32_t));
    m->full[h] = 1;
    m->val[h] = 0;
    m->used++;
    return &m->val[h];
}

static int vmap_grow(vmap *m)
{
    vmap n;
    if (vmap_alloc(&n, m->nv, m->cap * 2) != OR_OK) return OR_ENOMEM;
    for (uint64_t s = 0; s < m->cap; s++) {
        if (!m->full[s]) continue;
        const uint32_t *e = m->keys + s * m->nv;
        uint64_t h = hash_vec(e, n.nv) & (n.cap - 1);
        while (n.full[h]) h = (h + 1) & (n.cap - 1);
        memcpy(n.keys + h * n.nv, e, n.nv * sizeof(uint32_t));
        n.full[h] = 1;
        n.val[h] = m->val[s];
        n.used++;
    }
    vmap_free(m);
    *m = n;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* canonical operands and the error rules                              */
/* ------------------------------------------------------------------ */

typedef struct {
    uint32_t nv;
    uint64_t n;
    uint32_t *e; /* n * nv */
    i128 *c;
} cpoly;

static void cpoly_free(cpoly *p) { free(p->e); free(p->c); p->e = NULL; p->c = NULL; p->n = 0; }

static int check_packing(uint32_t nv, const uint8_t *w)
{
    if (nv < 1 || nv > 16 || !w) return OR_EINVAL;
    uint32_t sum = 0;
    for (uint32_t v = 0; v < nv; v++) {
        if (w[v] < 1 || w[v] > 32) return OR_EINVAL;
        sum += w[v];
    }
    return sum <= 64 ? OR_OK : OR_EINVAL;
}

/* Every exponent of an input term must leave the guard bit clear. */
static int check_inputs(uint32_t nv, const uint8_t *w, const uint32_t *exps, uint64_t n)
{
    for (uint64_t t = 0; t < n; t++)
        for (uint32_t v = 0; v < nv; v++)
            if ((uint64_t)exps[t * nv + v] >= ((uint64_t)1 << (w[v] - 1))) return OR_EEXP_OVERFLOW;
    return OR_OK;
}

/* Combine repeated monomials and drop zero coefficients. */
static int canonical(uint32_t nv, int kind, const uint32_t *exps, const void *coefs, uint64_t n,
                     cpoly *out)
{
    vmap m;
    out->nv = nv; out->n = 0; out->e = NULL; out->c = NULL;
    if (vmap_init(&m, nv, n) != OR_OK) return OR_ENOMEM;
    for (uint64_t t = 0; t < n; t++) {
        i128 *s = vmap_slot(&m, exps + t * nv);
        if (!s) { vmap_free(&m); return OR_ENOMEM; }
        *s = coef_add(kind, *s, coef_in(kind, coefs, t));
    }
    out->e = (uint32_t *)malloc((m.used + 1) * nv * sizeof(uint32_t));
    out->c = (i128 *)malloc((m.used + 1) * sizeof(i128));
    if (!out->e || !out->c) { vmap_free(&m); cpoly_free(out); return OR_ENOMEM; }
    int rc = OR_OK;
    for (uint64_t s = 0; s < m.cap; s++) {
        if (!m.full[s] || m.val[s] == 0) continue;
        if (kind == OR_KIND_I64 && (m.val[s] > (i128)INT64_MAX || m.val[s] < (i128)INT64_MIN))
            rc = OR_ECOEF_BOUND;
        memcpy(out->e + out->n * nv, m.keys + s * nv, nv * sizeof(uint32_t));
        out->c[out->n++] = m.val[s];
    }
    vmap_free(&m);
    if (rc != OR_OK) cpoly_free(out);
    return rc;
}

static u128 abs128(i128 x) { return x < 0 ? (u128)(-x) : (u128)x; }

/* Validation, canonical operands, exponent-sum and int128 bound checks. */
static int prepare(uint32_t nv, const uint8_t *w, int kind,
                   const uint32_t *fe, const void *fc, uint64_t nf,
                   const uint32_t *ge, const void *gc, uint64_t ng, cpoly *F, cpoly *G)
{
    int rc;
    F->e = G->e = NULL; F->c = G->c = NULL; F->n = G->n = 0;
    if ((rc = check_packing(nv, w)) != OR_OK) return rc;
    if (kind != OR_KIND_M61 && kind != OR_KIND_I64) return OR_EINVAL;
    if ((nf && (!fe || !fc)) || (ng && (!ge || !gc))) return OR_EINVAL;
    if ((rc = check_inputs(nv, w, fe, nf)) != OR_OK) return rc;
    if ((rc = check_inputs(nv, w, ge, ng)) != OR_OK) return rc;
    if ((rc = canonical(nv, kind, fe, fc, nf, F)) != OR_OK) return rc;
    if ((rc = canonical(nv, kind, ge, gc, ng, G)) != OR_OK) { cpoly_free(F); return rc; }
    if (F->n && G->n) {
        /* the largest exponent of x_v in the product is maxF_v + maxG_v */
        for (uint32_t v = 0; v < nv; v++) {
            uint64_t mf = 0, mg = 0;
            for (uint64_t i = 0; i < F->n; i++) if (F->e[i * nv + v] > mf) mf = F->e[i * nv + v];
            for (uint64_t j = 0; j < G->n; j++) if (G->e[j * nv + v] > mg) mg = G->e[j * nv + v];
            if (mf + mg >= ((uint64_t)1 << (w[v] - 1))) rc = OR_EEXP_OVERFLOW;
        }
        if (rc == OR_OK && kind == OR_KIND_I64) {
            u128 ma = 0, mb = 0;
            for (uint64_t i = 0; i < F->n; i++) if (abs128(F->c[i]) > ma) ma = abs128(F->c[i]);
            for (uint64_t j = 0; j < G->n; j++) if (abs128(G->c[j]) > mb) mb = abs128(G->c[j]);
            u128 mn = F->n < G->n ? F->n : G->n;
            u128 lim = ((((u128)1) << 127) - 1) / mn; /* ma*mb*mn >= 2^127 <=> ma*mb > lim */
            if (ma * mb > lim) rc = OR_ECOEF_BOUND;
        }
        if (rc != OR_OK) { cpoly_free(F); cpoly_free(G); }
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* lexicographic order on exponent vectors, x_1 most significant       */
/* ------------------------------------------------------------------ */

typedef struct { const uint32_t *e; uint32_t nv; } lexctx;

static int lex_cmp_idx(const void *a, const void *b, void *arg)
{
    const lexctx *c = (const lexctx *)arg;
    const uint32_t *x = c->e + (*(const uint64_t *)a) * c->nv;
    const uint32_t *y = c->e + (*(const uint64_t *)b) * c->nv;
#if ORACLE_PLANT == 5 /* planted mistake: x_n taken as the most significant variable */
    for (int v = (int)c->nv - 1; v >= 0; v--)
        if (x[v] != y[v]) return x[v] < y[v] ? -1 : 1;
    return 0;
#endif
    for (uint32_t v = 0; v < c->nv; v++)
        if (x[v] != y[v]) return x[v] < y[v] ? -1 : 1;
    return 0;
}

static int emit_sorted(uint32_t nv, int kind, const uint32_t *e, const i128 *c, uint64_t n,
                       uint32_t **h_exps, void **h_coefs, uint64_t *nh)
{
    uint64_t *idx = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    uint32_t *oe = (uint32_t *)malloc((n + 1) * nv * sizeof(uint32_t));
    void *oc = malloc((n + 1) * (kind == OR_KIND_M61 ? 8 : 16));
    if (!idx || !oe || !oc) { free(idx); free(oe); free(oc); return OR_ENOMEM; }
    for (uint64_t t = 0; t < n; t++) idx[t] = t;
    lexctx ctx = { e, nv };
    qsort_r(idx, n, sizeof(uint64_t), lex_cmp_idx, &ctx);
    for (uint64_t t = 0; t < n; t++) {
        memcpy(oe + t * nv, e + idx[t] * nv, nv * sizeof(uint32_t));
        coef_out(kind, c[idx[t]], oc, t);
    }
    free(idx);
    *h_exps = oe; *h_coefs = oc; *nh = n;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* oracle_mul: the definition                                          */
/* ------------------------------------------------------------------ */

int oracle_mul(uint32_t nv, const uint8_t *w, int kind,
               const uint32_t *fe, const void *fc, uint64_t nf,
               const uint32_t *ge, const void *gc, uint64_t ng,
               uint32_t **h_exps, void **h_coefs, uint64_t *nh)
{
    cpoly F, G;
    *h_exps = NULL; *h_coefs = NULL; *nh = 0;
    int rc = prepare(nv, w, kind, fe, fc, nf, ge, gc, ng, &F, &G);
    if (rc != OR_OK) return rc;

    vmap m;
    uint32_t gamma[16];
    if (vmap_init(&m, nv, F.n < 1024 && G.n < 1024 ? F.n * G.n : 1 << 20) != OR_OK) {
        cpoly_free(&F); cpoly_free(&G); return OR_ENOMEM;
    }
    for (uint64_t i = 0; i < F.n; i++) {
        for (uint64_t j = 0; j < G.n; j++) {
#if ORACLE_PLANT == 2 /* planted mistake (mutation tests only): a dropped term */
            if (j + 1 == G.n && i == 0) continue;
#endif
            for (uint32_t v = 0; v < nv; v++) gamma[v] = F.e[i * nv + v] + G.e[j * nv + v];
#if ORACLE_PLANT == 3 /* planted mistake: a wrong index */
            gamma[0] = F.e[i * nv + 0] + G.e[j * nv + (nv - 1)];
#endif
            i128 *s = vmap_slot(&m, gamma);
            if (!s) { rc = OR_ENOMEM; goto done; }
#if ORACLE_PLANT == 1 /* planted mistake: a wrong sign */
            *s = coef_add(kind, *s, kind == OR_KIND_M61 ? (i128)((P61 - (uint64_t)coef_mul(kind, F.c[i], G.c[j])) % P61)
                                                        : -coef_mul(kind, F.c[i], G.c[j]));
#elif ORACLE_PLANT == 4 /* planted mistake: a transposed operand */
            *s = coef_add(kind, *s, coef_mul(kind, F.c[i], G.c[i % G.n]));
#else
            *s = coef_add(kind, *s, coef_mul(kind, F.c[i], G.c[j]));
#endif
        }
    }
    {
        uint32_t *e = (uint32_t *)malloc((m.used + 1) * nv * sizeof(uint32_t));
        i128 *c = (i128 *)malloc((m.used + 1) * sizeof(i128));
        uint64_t n = 0;
        if (!e || !c) { free(e); free(c); rc = OR_ENOMEM; goto done; }
        for (uint64_t s = 0; s < m.cap; s++) {
            if (!m.full[s] || m.val[s] == 0) continue;
            memcpy(e + n * nv, m.keys + s * nv, nv * sizeof(uint32_t));
            c[n++] = m.val[s];
        }
        rc = emit_sorted(nv, kind, e, c, n, h_exps, h_coefs, nh);
        free(e); free(c);
    }
done:
    vmap_free(&m);
    cpoly_free(&F); cpoly_free(&G);
    return rc;
}

/* ------------------------------------------------------------------ */
/* oracle_coef_at: one monomial at a time                              */
/* ------------------------------------------------------------------ */

int oracle_coef_at(uint32_t nv, const uint8_t *w, int kind,
                   const uint32_t *fe, const void *fc, uint64_t nf,
                   const uint32_t *ge, const void *gc, uint64_t ng,
                   const uint32_t *gammas, uint64_t count, void *out)
{
    cpoly F, G;
    int rc = prepare(nv, w, kind, fe, fc, nf, ge, gc, ng, &F, &G);
    if (rc != OR_OK) return rc;
    vmap gm;
    if (vmap_init(&gm, nv, G.n) != OR_OK) { cpoly_free(&F); cpoly_free(&G); return OR_ENOMEM; }
    for (uint64_t j = 0; j < G.n; j++) {
        i128 *s = vmap_slot(&gm, G.e + j * nv);
        if (!s) { rc = OR_ENOMEM; goto done; }
        *s = G.c[j];
    }
    uint32_t beta[16];
    for (uint64_t k = 0; k < count; k++) {
        const uint32_t *gam = gammas + k * nv;
        i128 acc = 0;
        for (uint64_t i = 0; i < F.n; i++) {
            int ok = 1;
            for (uint32_t v = 0; v < nv; v++) {
                if (F.e[i * nv + v] > gam[v]) { ok = 0; break; }
                beta[v] = gam[v] - F.e[i * nv + v];
            }
            if (!ok) continue;
            i128 *b = vmap_find(&gm, beta);
            if (b) acc = coef_add(kind, acc, coef_mul(kind, F.c[i], *b));
        }
        coef_out(kind, acc, out, k);
    }
done:
    vmap_free(&gm);
    cpoly_free(&F); cpoly_free(&G);
    return rc;
}

/* ------------------------------------------------------------------ */
/* oracle_eval: p(r) mod 2^61 - 1                                      */
/* ------------------------------------------------------------------ */

static uint64_t m61_pow(uint64_t b, uint64_t e)
{
    uint64_t r = 1;
    b %= P61;
    while (e) {
        if (e & 1) r = m61_mul(r, b);
        b = m61_mul(b, b);
        e >>= 1;
    }
    return r;
}

uint64_t oracle_eval(uint32_t nv, int kind, const uint32_t *exps, const void *coefs, uint64_t n,
                     const uint64_t *r)
{
    uint64_t acc = 0;
    for (uint64_t t = 0; t < n; t++) {
        uint64_t c;
        if (kind == OR_KIND_M61) c = m61_of_u64(((const uint64_t *)coefs)[t]);
        else if (kind == OR_KIND_I64) c = m61_of_i128((i128)((const int64_t *)coefs)[t]);
        else {
            const uint64_t *q = (const uint64_t *)coefs + 2 * t;
            c = m61_of_i128((i128)(((u128)q[1] << 64) | q[0]));
        }
        for (uint32_t v = 0; v < nv; v++) c = m61_mul(c, m61_pow(r[v], exps[t * nv + v]));
        acc = m61_add(acc, c);
    }
    return acc;
}

void oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* Alg. 1 on CPU threads                                               */
/* ------------------------------------------------------------------ */

/* Packed exponents (Sec. 7): x_1 in the most significant field. */
static void field_offsets(uint32_t nv, const uint8_t *w, uint32_t *off)
{
    uint32_t s = 0;
    for (int v = (int)nv - 1; v >= 0; v--) { off[v] = s; s += w[v]; }
}

static uint64_t pack_vec(uint32_t nv, const uint32_t *off, const uint32_t *e)
{
    uint64_t k = 0;
    for (uint32_t v = 0; v < nv; v++) k |= (uint64_t)e[v] << off[v];
    return k;
}

typedef struct { uint64_t key; i128 coef; } term_t;

static int term_cmp(const void *a, const void *b)
{
    uint64_t x = ((const term_t *)a)->key, y = ((const term_t *)b)->key;
    return x < y ? -1 : (x > y);
}

static uint64_t grid_push(uint64_t *out, uint64_t cap, uint64_t n, uint64_t v)
{
    if (n < cap) out[n] = v;
    return n + 1;
}

/* Sec. 5: rows i = 1, 1+s_i, ... ; in each, columns from j0_i with step s_j;
 * alternate grid rows are shifted by floor(n_b / 2l); the last row and the
 * last column are sampled with the same steps.  Indices below are 1-based as
 * in the paper.  Steps are clamped to >= 1 for operands shorter than l. */
uint64_t oracle_grid(const uint64_t *alpha, uint64_t na, const uint64_t *beta, uint64_t nb,
                     uint32_t l, uint64_t *out, uint64_t cap)
{
    if (!na || !nb || !l) return 0;
    uint64_t si = na / l ? na / l : 1;
    uint64_t sj = nb / l ? nb / l : 1;
    uint64_t stagger = nb / (2 * (uint64_t)l);
    uint64_t n = 0;
    for (uint64_t i = 1; i <= na; i += si) {
        uint64_t j0 = 1 + (((i - 1) / si) % 2) * stagger;
        for (uint64_t j = j0; j <= nb; j += sj) n = grid_push(out, cap, n, alpha[i - 1] + beta[j - 1]);
    }
    for (uint64_t j = 1; j <= nb; j += sj) n = grid_push(out, cap, n, alpha[na - 1] + beta[j - 1]);
    for (uint64_t i = 1; i <= na; i += si) n = grid_push(out, cap, n, alpha[i - 1] + beta[nb - 1]);
    return n;
}

static int u64_cmp(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y);
}

typedef struct {
    int kind;
    const uint64_t *ak, *bk;
    const i128 *ac, *bc;
    uint64_t na, nb;
    const uint64_t *S;
    uint64_t ns;
    term_t **D;
    uint64_t *Dn;
    atomic_ulong next;
    atomic_int err;
} alg1_job;

/* FindEdge + MergeSort for the interval [S_k, S_{k+1}). */
static int alg1_interval(alg1_job *J, uint64_t k, uint64_t *lmin, uint64_t *lmax)
{
    const uint64_t lo = J->S[k], hi = J->S[k + 1];
    uint64_t jl = J->nb, jh = J->nb, cnt = 0;
    /* staircase: both edges only move left as the row index grows */
    for (uint64_t i = 0; i < J->na; i++) {
        while (jl > 0 && J->ak[i] + J->bk[jl - 1] >= lo) jl--;
        while (jh > 0 && J->ak[i] + J->bk[jh - 1] >= hi) jh--;
        lmin[i] = jl;
        lmax[i] = jh;
        cnt += jh - jl;
    }
    term_t *buf = (term_t *)malloc((cnt + 1) * sizeof(term_t));
    if (!buf) return OR_ENOMEM;
    uint64_t t = 0;
    for (uint64_t i = 0; i < J->na; i++)
        for (uint64_t j = lmin[i]; j < lmax[i]; j++) {
            buf[t].key = J->ak[i] + J->bk[j];
            buf[t].coef = coef_mul(J->kind, J->ac[i], J->bc[j]);
            t++;
        }
    qsort(buf, cnt, sizeof(term_t), term_cmp);
    uint64_t u = 0;
    for (uint64_t s = 0; s < cnt;) {
        uint64_t e = s;
        i128 c = 0;
        while (e < cnt && buf[e].key == buf[s].key) c = coef_add(J->kind, c, buf[e++].coef);
        if (c != 0) { buf[u].key = buf[s].key; buf[u].coef = c; u++; }
        s = e;
    }
    J->D[k] = buf;
    J->Dn[k] = u;
    return OR_OK;
}

static void *alg1_worker(void *arg)
{
    alg1_job *J = (alg1_job *)arg;
    uint64_t *lmin = (uint64_t *)malloc((J->na + 1) * sizeof(uint64_t));
    uint64_t *lmax = (uint64_t *)malloc((J->na + 1) * sizeof(uint64_t));
    if (!lmin || !lmax) { atomic_store(&J->err, OR_ENOMEM); free(lmin); free(lmax); return NULL; }
    for (;;) {
        uint64_t k = atomic_fetch_add(&J->next, 1);  /* dynamic scheduling */
        if (k + 1 >= J->ns) break;
        if (alg1_interval(J, k, lmin, lmax) != OR_OK) atomic_store(&J->err, OR_ENOMEM);
    }
    free(lmin); free(lmax);
    return NULL;
}

static int sort_packed(uint32_t nv, const uint32_t *off, const cpoly *p, uint64_t **keys, i128 **coefs)
{
    term_t *t = (term_t *)malloc((p->n + 1) * sizeof(term_t));
    *keys = (uint64_t *)malloc((p->n + 1) * sizeof(uint64_t));
    *coefs = (i128 *)malloc((p->n + 1) * sizeof(i128));
    if (!t || !*keys || !*coefs) { free(t); free(*keys); free(*coefs); return OR_ENOMEM; }
    for (uint64_t i = 0; i < p->n; i++) { t[i].key = pack_vec(nv, off, p->e + i * nv); t[i].coef = p->c[i]; }
    qsort(t, p->n, sizeof(term_t), term_cmp);
    for (uint64_t i = 0; i < p->n; i++) { (*keys)[i] = t[i].key; (*coefs)[i] = t[i].coef; }
    free(t);
    return OR_OK;
}

int oracle_mul_alg1(uint32_t nv, const uint8_t *w, int kind,
                    const uint32_t *fe, const void *fc, uint64_t nf,
                    const uint32_t *ge, const void *gc, uint64_t ng,
                    uint32_t l, uint32_t threads,
                    uint32_t **h_exps, void **h_coefs, uint64_t *nh, uint64_t *n_intervals)
{
    cpoly F, G;
    *h_exps = NULL; *h_coefs = NULL; *nh = 0;
    if (n_intervals) *n_intervals = 0;
    int rc = prepare(nv, w, kind, fe, fc, nf, ge, gc, ng, &F, &G);
    if (rc != OR_OK) return rc;
    if (!F.n || !G.n) {
        cpoly_free(&F); cpoly_free(&G);
        return emit_sorted(nv, kind, NULL, NULL, 0, h_exps, h_coefs, nh);
    }
    uint32_t off[16];
    field_offsets(nv, w, off);
    uint64_t *ak = NULL, *bk = NULL, *S = NULL, *Dn = NULL;
    i128 *ac = NULL, *bc = NULL;
    term_t **D = NULL;
    uint64_t ns = 0;
    if ((rc = sort_packed(nv, off, &F, &ak, &ac)) != OR_OK) goto out;
    if ((rc = sort_packed(nv, off, &G, &bk, &bc)) != OR_OK) goto out;

    /* first step: grid S*, gamma_end, sort, remove duplicates */
    {
        uint64_t cap = oracle_grid(ak, F.n, bk, G.n, l ? l : 1, NULL, 0) + 1;
        S = (uint64_t *)malloc(cap * sizeof(uint64_t));
        if (!S) { rc = OR_ENOMEM; goto out; }
        ns = oracle_grid(ak, F.n, bk, G.n, l ? l : 1, S, cap);
        S[ns++] = ak[F.n - 1] + bk[G.n - 1] + 1; /* gamma_end: exclusive upper end */
        qsort(S, ns, sizeof(uint64_t), u64_cmp);
        uint64_t u = 0;
        for (uint64_t s = 0; s < ns; s++)
            if (u == 0 || S[s] != S[u - 1]) S[u++] = S[s];
        ns = u;
    }

    /* second step: intervals in parallel */
    D = (term_t **)calloc(ns, sizeof(term_t *));
    Dn = (uint64_t *)calloc(ns, sizeof(uint64_t));
    if (!D || !Dn) { rc = OR_ENOMEM; goto out; }
    {
        alg1_job J;
        J.kind = kind; J.ak = ak; J.bk = bk; J.ac = ac; J.bc = bc; J.na = F.n; J.nb = G.n;
        J.S = S; J.ns = ns; J.D = D; J.Dn = Dn;
        atomic_init(&J.next, 0);
        atomic_init(&J.err, OR_OK);
        if (threads < 1) threads = 1;
        if (threads > 256) threads = 256;
        pthread_t tid[256];
        uint32_t started = 0;
        for (uint32_t t = 1; t < threads; t++)
            if (pthread_create(&tid[started], NULL, alg1_worker, &J) == 0) started++;
        alg1_worker(&J);
        for (uint32_t t = 0; t < started; t++) pthread_join(tid[t], NULL);
        if ((rc = atomic_load(&J.err)) != OR_OK) goto out;
    }
    if (n_intervals) *n_intervals = ns - 1;

    /* concatenate the containers in ascending interval order */
    {
        uint64_t total = 0;
        for (uint64_t k = 0; k + 1 < ns; k++) total += Dn[k];
        uint32_t *oe = (uint32_t *)malloc((total + 1) * nv * sizeof(uint32_t));
        void *oc = malloc((total + 1) * (kind == OR_KIND_M61 ? 8 : 16));
        if (!oe || !oc) { free(oe); free(oc); rc = OR_ENOMEM; goto out; }
        uint64_t t = 0;
        for (uint64_t k = 0; k + 1 < ns; k++)
            for (uint64_t q = 0; q < Dn[k]; q++, t++) {
                for (uint32_t v = 0; v < nv; v++) {
                    uint64_t mask = ((uint64_t)1 << w[v]) - 1;
                    oe[t * nv + v] = (uint32_t)((D[k][q].key >> off[v]) & mask);
                }
                coef_out(kind, D[k][q].coef, oc, t);
            }
        *h_exps = oe; *h_coefs = oc; *nh = total;
    }
out:
    if (D) for (uint64_t k = 0; k < ns; k++) free(D[k]);
    free(D); free(Dn); free(S);
    free(ak); free(bk); free(ac); free(bc);
    cpoly_free(&F); cpoly_free(&G);
    return rc;
}
