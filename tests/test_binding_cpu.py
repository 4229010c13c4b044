"""The binding's argument checks reject mis-shaped or mis-typed tensors before
any pointer reaches the library (no GPU needed: the checks look only at shapes
and element types, and come before the device checks)."""

import pytest
import torch

from paper_1303_7425_gb300 import _native as N


def _ops(nf=5, ng=7, nv=3):
    return (torch.zeros((nf, nv), dtype=torch.int32), torch.zeros(nf, dtype=torch.int64),
            torch.zeros((ng, nv), dtype=torch.int32), torch.zeros(ng, dtype=torch.int64))


def test_good_operands_and_outputs_pass():
    N.check_operands([8, 8, 8], *_ops())
    assert N.check_out((torch.zeros(11, dtype=torch.int64), torch.zeros(11, dtype=torch.int64)), "m61") == 11
    assert N.check_out((torch.zeros(11, dtype=torch.int64), torch.zeros((11, 2), dtype=torch.int64)), "i64") == 11
    assert N.check_out((torch.zeros(4, dtype=torch.int64), torch.zeros((4, 3), dtype=torch.int64)), "i192") == 4


@pytest.mark.parametrize("case", ["nvars", "exps_dtype", "coef_len", "coef_dtype", "coef_2d"])
def test_bad_operands_rejected(case):
    fe, fc, ge, gc = _ops()
    if case == "nvars":
        fe = torch.zeros((5, 2), dtype=torch.int32)
    elif case == "exps_dtype":
        ge = ge.to(torch.int64)
    elif case == "coef_len":
        gc = torch.zeros(6, dtype=torch.int64)
    elif case == "coef_dtype":
        fc = fc.to(torch.int32)
    elif case == "coef_2d":
        fc = torch.zeros((5, 1), dtype=torch.int64)
    with pytest.raises(ValueError):
        N.check_operands([8, 8, 8], fe, fc, ge, gc)


@pytest.mark.parametrize("kind,coef_shape", [("i64", (9,)), ("m61", (9, 2)), ("i64", (9, 3)), ("i192", (9, 2)),
                                             ("m61", (8,))])
def test_bad_output_word_count_rejected(kind, coef_shape):
    """An int128 result needs two words per term: a (cap,) tensor would let
    the kernel write past the end of the caller's allocation."""
    with pytest.raises(ValueError):
        N.check_out((torch.zeros(9, dtype=torch.int64), torch.zeros(coef_shape, dtype=torch.int64)), kind)


def test_bad_output_dtype_rejected():
    with pytest.raises(ValueError):
        N.check_out((torch.zeros(9, dtype=torch.int32), torch.zeros(9, dtype=torch.int64)), "m61")
    with pytest.raises(ValueError):
        N.check_out((torch.zeros(9, dtype=torch.int64), torch.zeros(9, dtype=torch.float64)), "m61")


def test_entry_points_check_shapes_before_the_device():
    """The public calls run the shape checks first, so a CPU run sees the
    shape error, not the missing-device error."""
    fe, fc, ge, gc = _ops()
    bad_out = (torch.zeros(9, dtype=torch.int64), torch.zeros(9, dtype=torch.int64))
    with pytest.raises(ValueError, match="kind 'i64'"):
        N.polymul_noalloc([8, 8, 8], fe, fc, ge, gc, bad_out, kind="i64")
    with pytest.raises(ValueError, match="kind 'i64'"):
        N.Plan([8, 8, 8], fe, fc, ge, gc, bad_out, kind="i64")
    with pytest.raises(ValueError, match="f_exps"):
        N.polymul([8, 8], fe, fc, ge, gc)
    with pytest.raises(ValueError, match="kind 'i64'"):
        N._batch_item(dict(field_bits=[8, 8, 8], kind="i64", f_exps=fe, f_coefs=fc, g_exps=ge, g_coefs=gc,
                           out=bad_out))
