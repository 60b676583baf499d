"""The planner's default launch configuration.  Without a tuning entry a plan
takes the dtype pair's first compiled shape at that shape's stored CTAs per
SM (as many as fit when the shape names none); an explicit CTA count in the
descriptor is taken as given, and a count above what fits is lowered to it.
The checks read the configuration back through sepconv5_plan_info; which
configuration is fastest is measured by the autotuner and the bench, not
asserted here."""
import pytest

pytestmark = pytest.mark.gpu

H = W = 4096


@pytest.fixture(scope="module")
def sc5():
    from paper_1711_09791_gb300 import sepconv5
    sepconv5.load()
    sepconv5.autotune(0, [])  # no tuning table: the defaults apply
    return sepconv5


def _info(sc5, dtype, out_dtype=None, **kw):
    p = sc5.Plan(3, H, W, W, W - 4, dtype, out_dtype, **kw)
    try:
        return p.info()
    finally:
        p.close()


@pytest.mark.parametrize("dtype,out_dtype,ctas", [("bf16", "bf16", 2), ("f16", "f16", 2)])
def test_untuned_plan_takes_the_default_shape_and_count(sc5, dtype, out_dtype, ctas):
    th, tw, st = sc5.fused_configs(dtype, out_dtype)[0]
    info = _info(sc5, dtype, out_dtype)
    assert (info["tile_h"], info["tile_w"], info["stages"]) == (th, tw, st)
    # the 16-bit default shape stores 2 CTAs per SM (its measured best on 3 x 8192^2)
    assert info["ctas_per_sm"] == ctas


def test_untuned_f32_plan_fills_the_sm(sc5):
    th, tw, st = sc5.fused_configs("f32")[0]
    info = _info(sc5, "f32")
    assert (info["tile_h"], info["tile_w"], info["stages"]) == (th, tw, st)
    # the FP32 default names no count: as many as fit, and at least one
    fit = _info(sc5, "f32", ctas_per_sm=64)["ctas_per_sm"]
    assert 1 <= info["ctas_per_sm"] == fit


def test_explicit_count_is_taken_and_capped(sc5):
    th, tw, st = sc5.fused_configs("bf16")[0]
    one = _info(sc5, "bf16", tile_h=th, tile_w=tw, stages=st, ctas_per_sm=1)
    assert (one["tile_h"], one["stages"], one["ctas_per_sm"]) == (th, st, 1)
    many = _info(sc5, "bf16", tile_h=th, tile_w=tw, stages=st, ctas_per_sm=64)
    assert 1 <= many["ctas_per_sm"] < 64
