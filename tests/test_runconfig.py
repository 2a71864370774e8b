"""Per-run JSON configuration: defaults, validation and the mapping onto gsw_solver_opts (CPU)."""
import json

import pytest

from paper_2404_17754_gb300 import gsw, runconfig


def test_defaults_and_file_round_trip(tmp_path):
    cfg = runconfig.resolve({})
    assert cfg == runconfig.DEFAULTS and cfg is not runconfig.DEFAULTS
    path = tmp_path / "run.json"
    path.write_text(json.dumps({"workload": {"kind": "realistic", "crop": 12, "directions": [2, 0]},
                                "solver": {"precision": "fp16", "coarse_weight": 1.0, "coarse_relres": 1e-5}}))
    cfg = runconfig.resolve(str(path))
    assert cfg["workload"]["kind"] == "realistic" and cfg["workload"]["directions"] == [2, 0]
    assert cfg["solver"]["tol"] == 1e-8  # untouched keys keep their defaults
    json.dumps(cfg)  # the resolved configuration is itself JSON


@pytest.mark.parametrize("bad", [
    {"solvr": {}},
    {"solver": {"toll": 1e-8}},
    {"solver": {"precision": "fp8"}},
    {"solver": {"outer_op": "fp128"}},
    {"workload": {"kind": "octree"}},
    {"workload": {"directions": []}},
    {"workload": {"directions": [0, 0]}},
    {"workload": {"directions": [3]}},
    {"time": {"n_steps": 0}},
    {"time": {"band": [5.0, 0.5]}},
    {"solver": 3},
    [],
])
def test_invalid_configurations_are_rejected(bad):
    with pytest.raises(ValueError):
        runconfig.resolve(bad)


def test_solver_section_covers_the_option_struct():
    """Every field of gsw_solver_opts except the host-driven scheduling knobs (check_every,
    inner_variant: left to the library's defaults and autotuner) comes from the configuration."""
    kw = runconfig.solver_kwargs(runconfig.resolve({"solver": {"precision": "fp32", "outer_op": "dword"}}))
    fields = {name for name, _ in gsw.SolverOpts._fields_}
    assert set(kw) == fields - {"check_every", "inner_variant"}
    assert kw["precision"] == gsw.PREC_FP32 and kw["outer_op"] == 2
