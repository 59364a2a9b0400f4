"""Host-side checks of the CUDA library (no GPU needed): exported symbols, the basis-function
table against the oracle's (bit-exact), FoM band assignment, argument validation."""
import ctypes
import re

import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O
from paper_2412_17617_gb300 import build as B
from paper_2412_17617_gb300 import pmom


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pmom.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(B.PUBLIC_HEADER).read()
    declared = set(re.findall(r"^(?:pmom_status|const char\*)\s+(pmom_\w+)\(", hdr, re.M))
    assert declared == set(pmom.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def _grids():
    gs = [PI.grid_plain_8x8(), PI.grid_stripline_16x16x2(), PI.grid_tiny(3), PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2),
          PI.grid_stripline_32x32x4()]
    # every port side, several positions, non-square grid
    ports = (PI.Port(0, 0, 0), PI.Port(0, 1, 4), PI.Port(1, 2, 2), PI.Port(1, 3, 0))
    gs.append(PI.Grid("sides_5x3x2", 2, 5, 3, 1e-3, PI.MEDIUM_STRIPLINE, (0.5e-3, 1.0e-3), 1.5e-3, 3.66, 0.004, 2,
                      ports))
    # three-state grids (via BFs after the pixel-port BFs)
    gs.append(PI.Grid("sides_5x3x2_via", 2, 5, 3, 1e-3, PI.MEDIUM_STRIPLINE, (0.5e-3, 1.0e-3), 1.5e-3, 3.66, 0.004, 3,
                      ports))
    gs.append(PI.grid_stripline_20x20x3(n_states=3))
    # uniform and random diagonal orientations
    import dataclasses
    gs.append(dataclasses.replace(PI.grid_stripline_16x16x2(), name="stripline_16x16x2_uniform", diag_pattern=1))
    gs.append(dataclasses.replace(gs[-3], name="sides_5x3x2_via_random", diag_pattern=2, diag_seed=77))
    # 8- and 18-triangle pixels (multi-edge port gaps), with every orientation pattern
    gs.append(dataclasses.replace(PI.grid_tiny(3), name="tiny_s2", sub=2))
    gs.append(dataclasses.replace(PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2), name="strip_s3_random", sub=3,
                                  diag_pattern=2, diag_seed=5))
    gs.append(dataclasses.replace(gs[5], name="sides_5x3x2_s2_uniform", sub=2, diag_pattern=1))
    return gs


@pytest.mark.parametrize("g", _grids(), ids=lambda g: g.name)
def test_bf_table_bit_exact_vs_oracle(lib, g):
    ev = pmom.Evaluator(g)
    ours = ev.bf_table()
    ref = O.Grid(g).table
    assert ours.shape == ref.shape
    assert np.array_equal(ours, ref)
    ev.close()


@pytest.mark.parametrize("w", [PI.workload_plain(), PI.workload_precision()], ids=lambda w: w.name)
def test_band_codes_match_oracle(w):
    assert np.array_equal(pmom.band_codes(w.freqs(), w.bands), O.bands(w.freqs(), w.bands))


def test_argument_validation(lib):
    g = PI.grid_tiny(3)
    bad = PI.Grid("bad", 1, 3, 3, 1e-3, 0, (0.5e-3,), 0.5e-3, 3.5, 0.0, 2, (PI.Port(0, 0, 7),))
    with pytest.raises(pmom.PmomError) as e:
        pmom.Evaluator(bad)
    assert e.value.status == 1
    # a via needs a layer above it
    three = PI.Grid("via", 1, 3, 3, 1e-3, 0, (0.5e-3,), 0.5e-3, 3.5, 0.0, 3, (PI.Port(0, 0, 1),))
    with pytest.raises(pmom.PmomError) as e:
        pmom.Evaluator(three)
    assert e.value.status == 1
    pat = PI.Grid("pattern", 1, 3, 3, 1e-3, 0, (0.5e-3,), 0.5e-3, 3.5, 0.0, 2, (PI.Port(0, 0, 1),), diag_pattern=3)
    with pytest.raises(pmom.PmomError) as e:
        pmom.Evaluator(pat)
    assert e.value.status == 1
    # 2, 8 or 18 triangles per pixel; a via needs the two-triangle pixel
    import dataclasses
    for bad_grid in (dataclasses.replace(g, sub=4),
                     dataclasses.replace(PI.grid_stripline_20x20x3(n_states=3), sub=2)):
        with pytest.raises(pmom.PmomError) as e:
            pmom.Evaluator(bad_grid)
        assert e.value.status == 1
    # the layered microstrip's kernels are those of horizontal currents: no via state there
    pmom.Evaluator(dataclasses.replace(g, medium=2)).close()
    with pytest.raises(pmom.PmomError) as e:
        pmom.Evaluator(dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_MICROSTRIP, 2), medium=2, n_states=3))
    assert e.value.status == 7
    four = PI.Grid("four", 2, 3, 3, 1e-3, 0, (0.5e-3, 1e-3), 1e-3, 3.5, 0.0, 4, (PI.Port(0, 0, 1),))
    with pytest.raises(pmom.PmomError) as e:
        pmom.Evaluator(four)
    assert e.value.status == 7
    ev = pmom.Evaluator(g)
    with pytest.raises(pmom.PmomError) as e:
        ev.set_fom(np.zeros(2, np.uint8))
    assert e.value.status == 6   # NOT_READY: no database yet
    st = lib.pmom_eval_candidates(ev.h, ctypes.c_void_p(1), 4, 1, None, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert st == 6
    st = lib.pmom_eval_candidates(ev.h, None, 4, 1, None, None, None, None)
    assert st == 1
    ev.close()


def test_search_rejects_depth_beyond_the_column_count(lib):
    """pmom_search on a 2 x 2 grid (four columns) with d_max = 8: INVALID_ARG before any
    evaluation, where a deeper tree would have no free column to draw."""
    g = PI.grid_tiny(2)
    ev = pmom.Evaluator(g)
    init = PI.seed_map(g, 0.5, 1)
    for call in (ev.search, ev.search_resume):
        with pytest.raises(pmom.PmomError) as e:
            call(init, seed=1, d_max=8, m_of_d=(1,) * 8, max_evals=10)
        assert e.value.status == 1
    ev.close()


def test_phase_profiler_names_match_kernel_slots():
    """The profiler's phase names follow the kernel's phase-slot enum in order (the profiling build
    reports cycles by slot index)."""
    import os
    import re
    from paper_2412_17617_gb300 import phases
    src = open(os.path.join(os.path.dirname(phases.__file__), "csrc", "pmom_eval_kernels.cuh")).read()
    body = re.search(r"enum Phase : int \{(.*?)\};", src, re.S).group(1)
    slots = {name: int(v) for name, v in re.findall(r"(kPh\w+)\s*=\s*(\d+)", body)}
    assert sorted(slots.values()) == list(range(len(slots)))
    assert len(phases.NAMES) == len(slots)
    assert slots["kPhTasks"] == phases.TASKS
    order = [n for n, _ in sorted(slots.items(), key=lambda kv: kv[1])]
    expect = {"kPhGather": "gather", "kPhLu": "lu", "kPhResid": "resid", "kPhPanelFactor": "panelfactor",
              "kPhColGemm": "colgemm", "kPhRowGemm": "rowgemm", "kPhInnerUpd": "innerupd", "kPhGemmConv": "g_conv"}
    for k, n in expect.items():
        assert phases.NAMES[order.index(k)] == n
