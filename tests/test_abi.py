"""The C ABI without a GPU: the library builds, loads, exports every symbol that
include/stage.h declares, and the ctypes structures match the C layouts."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stage.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_05291_gb300 import build
    return build.build()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^STAGE_API\s+[\w\s\*]+?\b(stage_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("stage_create", "stage_destroy", "stage_load_instance", "stage_rank_bases",
                 "stage_evaluate_placement", "stage_tabu_run"):
        assert must in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    # nothing that could interpose libc (an exported bare `poll` would)
    assert "poll" not in exported


def test_library_loads_and_binds(libpath):
    from paper_2001_05291_gb300 import stage
    L = stage.lib()
    assert L.stage_version() >= 10000
    for n in declared_symbols():
        assert hasattr(L, n)


LAYOUT_PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "stage.h"
#define P(T) printf(#T " %zu\n", sizeof(T))
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  P(stage_config); O(stage_config, spin_limit); O(stage_config, alloc); O(stage_config, stream);
  P(stage_instance_desc); O(stage_instance_desc, base_xy); O(stage_instance_desc, base_available);
  P(stage_move); O(stage_move, cov);
  P(stage_tabu_state); O(stage_tabu_state, open); O(stage_tabu_state, tabu_expiry);
  P(stage_tabu_params); O(stage_tabu_params, start_open); O(stage_tabu_params, resume);
  P(stage_tabu_result); O(stage_tabu_result, best_open); O(stage_tabu_result, end_state);
  P(stage_update); O(stage_update, add_pick_xy); O(stage_update, avail_ids);
  P(stage_request); O(stage_request, params); O(stage_request, traj); O(stage_request, final_open);
  O(stage_request, resume_resident);
  P(stage_result); O(stage_result, n_forced); O(stage_result, best_cov); O(stage_result, t_end_ns);
  P(stage_ls_params); O(stage_ls_params, perm_slots); O(stage_ls_params, start_open);
  P(stage_ls_result); O(stage_ls_result, final_cov); O(stage_ls_result, final_open);
  P(stage_fleet_params); O(stage_fleet_params, base_helipad); O(stage_fleet_params, start_fixed);
  P(stage_fleet_result); O(stage_fleet_result, final_dist); O(stage_fleet_result, final_fixed);
  return 0;
}
"""


def test_ctypes_layouts_match_header(tmp_path):
    import ctypes
    from paper_2001_05291_gb300 import stage
    src = tmp_path / "probe.c"
    src.write_text(LAYOUT_PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.splitlines())
    py = {"stage_config": stage.StageConfig, "stage_instance_desc": stage.StageInstanceDesc,
          "stage_move": stage.StageMove, "stage_tabu_state": stage.StageTabuState,
          "stage_tabu_params": stage.StageTabuParams, "stage_tabu_result": stage.StageTabuResult,
          "stage_update": stage.StageUpdate, "stage_request": stage.StageRequest,
          "stage_result": stage.StageResult, "stage_ls_params": stage.StageLsParams,
          "stage_ls_result": stage.StageLsResult, "stage_fleet_params": stage.StageFleetParams,
          "stage_fleet_result": stage.StageFleetResult}
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(py[t], f).offset == int(val), key
        else:
            assert ctypes.sizeof(py[key]) == int(val), key


def test_create_without_gpu_fails_loudly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2001_05291_gb300 import stage
    with pytest.raises(stage.StageError) as e:
        stage.Context(device=0, torch_memory=False)
    assert e.value.status == -6   # STAGE_ERR_CUDA: no CPU fallback


def test_binding_constants_match_header():
    """The binding's flag and status values are the header's #defines."""
    from paper_2001_05291_gb300 import stage
    with open(HEADER) as fh:
        defs = dict(re.findall(r"#define\s+(STAGE_[A-Z_0-9]+)\s+\(?(-?\d+)u?\)?", fh.read()))
    names = ["STAGE_THREADSAFE", "STAGE_PROFILE", "STAGE_AUTOTUNE", "STAGE_FULL_PASS", "STAGE_INCREMENTAL",
             "STAGE_NO_PERSIST", "STAGE_DESC_HAVERSINE"]
    for n in names:
        assert n in defs, n
        assert getattr(stage, n) == int(defs[n]), n
    flags = [int(defs[n]) for n in names[:6]]
    assert len(set(flags)) == 6 and all(f & (f - 1) == 0 for f in flags)   # distinct single bits
