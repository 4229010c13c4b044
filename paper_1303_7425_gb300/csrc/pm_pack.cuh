// K-a interface: packing and operand canonicalisation (pm_pack.cu).
#pragma once

#include "pm_common.cuh"

namespace pm {

// A canonical operand on the device: sorted by monomial order, distinct
// monomials, no zero coefficient.  key = packed guard-bit key, rank = the
// monomial's mixed-radix rank in the product's exponent box, coef = residue
// mod p (M61) or int64 bits (I64).
struct Operand {
    u64 n = 0;
    u64 *key = nullptr;
    u64 *rank = nullptr;
    u64 *coef = nullptr;
};

void input_maxima(Ctx &c, const pm_terms_in &in, const Layout &L, u32 *d_maxe, u32 *d_status);
void canonicalize(Ctx &c, Scratch &S, const pm_terms_in &in, const Layout &raw, u64 raw_box, int kind,
                  Operand &op, u32 *d_status, u64 *d_count);
// Canonical operand by scatter into its own exponent box (own_box slots,
// strides in `own`): for boxes not much larger than the operand.
void canonicalize_dense(Ctx &c, Scratch &S, const pm_terms_in &in, const Layout &own, u64 own_box, int kind,
                        Operand &op, u32 *d_status, u64 *d_count,
                        const u32 *abort = nullptr);
void operand_stats(Ctx &c, const Operand &op, u64 n_max, const u64 *d_n, const Layout &L, int kind, u32 *d_maxe,
                   u64 *d_maxabs, u64 *d_first_last);
// rank32 (optional): also store the low 32 bits of each rank
void operand_ranks(Ctx &c, Operand &op, const Layout &L, u32 *rank32 = nullptr);
void pack_keys(Ctx &c, const u32 *exps, size_t n, const Layout &L, u64 *keys, u32 *d_status);
void unpack_keys(Ctx &c, const u64 *keys, size_t n, const Layout &L, u32 *exps);

}  // namespace pm
