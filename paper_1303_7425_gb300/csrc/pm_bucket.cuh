// Bucketed sort strategy interface (pm_bucket.cu).
#pragma once

#include <vector>

#include "pm_common.cuh"

namespace pm {

struct BucketInputs {
    const u64 *A, *Ac;  // canonical f: sorted keys, coefficients (mod p residues or int64)
    const u64 *B, *Bc;  // canonical g
    u32 na, nb;
    u64 A_last, B_last;  // the last (largest) keys of f and g
};

// The result as slices for the compaction: bucket k's terms start at
// key[base[k]] (coefficients at coef[words * base[k]]) and number ucount[k].
struct BucketSlices {
    u64 n = 0;           // buckets
    u64 *key = nullptr, *coef = nullptr;
    const u64 *base = nullptr, *ucount = nullptr;
    u32 words = 1;
    u32 big = 0;         // buckets sorted outside shared memory
};

// h's terms with keys in [lo, end); kind PM_COEF_M61 or PM_COEF_I64_ACC128.
BucketSlices bucket_product(Ctx &c, Scratch &S, const BucketInputs &in, int kind, u64 lo, u64 end, u64 products);

}  // namespace pm
