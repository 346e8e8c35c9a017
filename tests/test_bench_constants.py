"""bench.py's algorithmic-flop constants agree with the flop-counting oracle
and with the stored tests/golden/flops_per_unit.json."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(path, name):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def counts():
    gen = _load(os.path.join(HERE, "golden", "make_flop_counts.py"), "make_flop_counts")
    return gen.count()


def test_stored_counts_are_current(counts):
    stored = json.load(open(os.path.join(HERE, "golden", "flops_per_unit.json")))
    for k in ("per_zone_cycle", "flux_per_face", "recon_per_cell_dir", "update_per_cell_stage"):
        assert abs(stored[k] - counts[k]) <= 1e-9 * counts[k], k


def test_bench_constants_match(counts):
    bench = _load(os.path.join(os.path.dirname(HERE), "bench.py"), "bench_mod")
    pairs = [(bench.FLOPS_PER_FACE, counts["flux_per_face"]),
             (bench.FLOPS_PER_RECON_CELL, counts["recon_per_cell_dir"]),
             (bench.FLOPS_PER_UPDATE_CELL, counts["update_per_cell_stage"]),
             (bench.FLOPS_PER_ZONE_CYCLE, counts["per_zone_cycle"])]
    for have, want in pairs:
        assert abs(have - want) <= 1e-3 * want, (have, want)
