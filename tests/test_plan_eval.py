"""The planner's tables evaluated on the host (numpy) against the oracle, for
every channel id, upper and lower components (CPU: no GPU involved).

`bbc_plan_export` returns the block rows, block-pair tasks and signed sums
the CUDA kernels run; `plan_eval` runs them in numpy.  L = 3 is odd, so
q and -q differ for every q but 0 (a q / -q slip in a task would show);
the propagators are isospin-symmetric (S_u = S_d), as the plan assumes.
"""
import numpy as np
import pytest

import plan_eval
import synth
import oracle.oracle as orc
from paper_1510_00903_gb300 import bbc

L = 3


@pytest.fixture(scope="module")
def slice3():
    F = synth.flavour_set(L, 1, seed=81, isospin=True)
    return F["u"][0].copy(), F["s"][0].copy()


def _check(chans, components, S, tol=1e-12):
    Sl, Ss = S
    ctx = bbc.bbc_create_components(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, chans, components)
    try:
        plan = bbc.bbc_plan_export(ctx)
    finally:
        bbc.bbc_destroy(ctx)
    lower = components == bbc.BBC_LOWER
    got = plan_eval.correlator(plan, L, Sl, Ss, spin_offset=2 if lower else 0)
    want = orc.correlator(L, Sl, Sl, Ss, chans, lower=lower)
    ref = np.abs(want).reshape(len(chans), -1).max(axis=1)
    # channels that vanish identically (the four omitted ones in the isospin limit)
    # are compared against the largest correlator of the list
    scale = np.where(ref > 1e-9 * ref.max(), ref, ref.max())
    err = np.abs(got - want).reshape(len(chans), -1).max(axis=1) / scale
    assert err.max() < tol, (err.max(), chans[int(err.argmax())])


@pytest.mark.parametrize("components", [bbc.BBC_UPPER, bbc.BBC_LOWER])
def test_octet_and_charge_states(slice3, components):
    _check(list(range(64)), components, slice3)


@pytest.mark.parametrize("components", [bbc.BBC_UPPER, bbc.BBC_LOWER])
def test_decuplet(slice3, components):
    _check(list(range(64, 154)), components, slice3)


@pytest.mark.parametrize("components", [bbc.BBC_UPPER, bbc.BBC_LOWER])
@pytest.mark.parametrize("ids", [bbc.DELTA_DELTA + bbc.P_DELTA, bbc.SIGMA_STAR_PAIRS, bbc.XI_STAR_PAIRS],
                         ids=["Delta++ and p Delta++", "Sigma*+ pairs", "Xi*0 pairs"])
def test_decuplet_families(slice3, components, ids):
    """The (l, l), (l, s) and (s, l) vector diquarks, the two-term operators
    (one term's eps over an odd reordering of its quark string) and the
    (s, l) -> (l, s) slot swap of a symmetric diquark matrix."""
    _check(ids, components, slice3)


def test_single_channel_plans(slice3):
    """Plans of one channel (other block sets, families and diquark lists)."""
    for ch in (0, 1, 10, 37, 51, 60, 64, 121, 150):
        _check([ch], bbc.BBC_UPPER, slice3)


def test_plans_whose_products_all_vanish(slice3):
    """The four channels the paper omits cancel exactly in the isospin limit:
    their plans keep no block-pair task and no signed term, and evaluate to
    zero (as the oracle does with S_u = S_d)."""
    Sl, Ss = slice3
    ctx = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [52, 53, 54, 55])
    try:
        plan = bbc.bbc_plan_export(ctx)
    finally:
        bbc.bbc_destroy(ctx)
    assert len(plan["tasks"]) == 0 and len(plan["items"]) == 0
    got = plan_eval.correlator(plan, L, Sl, Ss)
    want = orc.correlator(L, Sl, Sl, Ss, [52, 53, 54, 55])
    ref = np.abs(orc.correlator(L, Sl, Sl, Ss, [10])).max()
    assert np.abs(got).max() == 0 and np.abs(want).max() < 1e-13 * ref


def test_export_sizes_and_bounds():
    ctx = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, list(range(52)))
    try:
        p = bbc.bbc_plan_export(ctx)
        s = bbc.bbc_plan_sizes(ctx)
    finally:
        bbc.bbc_destroy(ctx)
    assert len(p["row_ptr"]) - 1 == s["block_outputs"] == 7368
    assert len(p["terms"]) == 33816 and 16 * len(p["tasks"]) == s["pair_items"]
    assert len(p["out_ptr"]) - 1 == 52 * 16
    assert p["terms"][:, 0].min() >= 0 and p["terms"][:, 0].max() <= 3  # octet families only
    assert p["terms"][:, 1].min() >= 0 and p["terms"][:, 1].max() < 2 * 1728
    assert np.all(p["terms"][:, 2] != 0)
    assert p["items"].max() < s["pair_items"]
