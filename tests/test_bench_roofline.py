"""The roofline arithmetic of bench.py's default line, on CPU.

dominant_roofline picks the stage with the most time among those with a
byte model, and reports achieved = bytes per unit x units per launch /
its time, frac = achieved / peak, and, where a DRAM figure per unit from an
ncu capture exists for that stage and precision, traffic = that figure x
units per launch and frac_traffic = traffic / time / peak."""
import math

import bench


def stages(deposit_ms, blocks_ms):
    K = 20
    ms = {k: 0.0 for k in bench.STAGES}
    ms.update({"deposit": deposit_ms, "blocks": blocks_ms, "photons": 1.5, "field": 3.1, "constants": 0.26,
               "end": 1.0})
    units = {"photons": 1.5e9, "blocks": 1.68e9, "deposit": 1.68e9, "massive": 1e5, "field": 512 ** 3 * K,
             "constants": 512 ** 3 * K}
    return {"steps": K, "ms_per_step": sum(ms.values()), "stage_ms": ms, "stage_units": units,
            "stage_bytes": {k: bench.STAGE_BYTES[k][0] for k in bench.STAGE_BYTES}, "precision": 32}


def test_longest_stage_with_its_bytes_and_traffic():
    rr = stages(4.6, 4.4)
    r = bench.dominant_roofline(rr, 6800.0, "measured")
    assert r["stage"] == "deposit" and r["bytes_per_unit"] == 48
    units = 1.68e9 / 20
    assert math.isclose(r["units_per_launch"], units)
    assert math.isclose(r["achieved"], 48 * units / 4.6e-3 / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / 6800.0)
    dram = bench.LARGE_DRAM_BYTES_PER_UNIT[("deposit", 32)]
    assert math.isclose(r["traffic"], dram * units)
    assert math.isclose(r["frac_traffic"], dram * units / 4.6e-3 / 1e9 / 6800.0)
    assert math.isclose(r["share_of_step"], 4.6 / rr["ms_per_step"])


def test_other_stage_and_no_traffic_figure():
    rr = stages(4.0, 4.4)
    r = bench.dominant_roofline(rr, 6800.0, "measured")
    assert r["stage"] == "blocks" and r["bytes_per_unit"] == 68
    # FP64 has no DRAM figure: traffic is null
    rr["precision"] = 64
    rr["stage_bytes"] = {k: bench.STAGE_BYTES[k][1] for k in bench.STAGE_BYTES}
    r = bench.dominant_roofline(rr, 6800.0, "measured")
    assert r["traffic"] is None and "frac_traffic" not in r and r["bytes_per_unit"] == 120
