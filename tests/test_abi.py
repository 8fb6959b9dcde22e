"""The C-ABI library loads and exports every entry point that include/*.h
declares; configuration errors are reported before any device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gaps_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_19633_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gaps_init", "gaps_generate_hard", "gaps_shower", "gaps_observables",
                     "gaps_get_stats", "gaps_error_string", "gaps_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_exports(lib):
    from paper_2511_19633_gb300 import gaps as G
    for name in declared_functions():
        assert name in G.EXPORTS and callable(getattr(G, name))


def test_error_strings(lib):
    from paper_2511_19633_gb300 import gaps as G
    assert G.gaps_error_string(0) == "ok"
    assert "capacity" in G.gaps_error_string(-2)
    assert G.gaps_error_string(12345) == "unknown error"


@pytest.mark.parametrize("field,value", [("process", 7), ("sqrt_s", -1.0), ("t_cut", 0.1),
                                         ("nmax_partons", 2), ("nmax_partons", 1000), ("nf", 9),
                                         ("block_size", 48), ("p_s", 1.5), ("schedule", 5),
                                         ("alpha_s_mz", 2.0), ("schedule", 3), ("wave_passes", -1),
                                         ("wave_passes", 5000), ("max_cycles", -5)])
def test_invalid_configuration_is_rejected_without_a_device(lib, pdf, field, value):
    from paper_2511_19633_gb300 import gaps as G
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf)
    setattr(cfg, field, value)
    with pytest.raises(G.GapsError) as e:
        G.gaps_init(cfg)
    assert e.value.code == G.GAPS_ERR_INVALID_ARG


def test_missing_pdf_is_rejected(lib):
    from paper_2511_19633_gb300 import gaps as G
    cfg = G.make_config(1, 13600.0, pdf_grid=None)
    with pytest.raises(G.GapsError) as e:
        G.gaps_init(cfg)
    assert e.value.code == G.GAPS_ERR_INVALID_ARG


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a small C program compiled with gcc."""
    import subprocess
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gaps.h"', 'int main(void) {',
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    return out[0], out[1:]


@pytest.mark.parametrize("struct,cls", [("gaps_config", "GapsConfig"), ("gaps_events", "GapsEvents"),
                                        ("gaps_stats", "GapsStats"), ("gaps_mix_row", "GapsMixRow"),
                                        ("gaps_hists", "GapsHists"), ("gaps_learn_config", "GapsLearnConfig"),
                                        ("gaps_learn_report", "GapsLearnReport")])
def test_binding_structs_match_the_header_layout(struct, cls, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of
    the C declaration (fields appended to the ABI must be appended in both)."""
    from paper_2511_19633_gb300 import gaps as G
    py = getattr(G, cls)
    names = [f[0] for f in py._fields_]
    size, offsets = _c_layout(struct, names, tmp_path)
    assert ctypes.sizeof(py) == size
    for name, off in zip(names, offsets):
        assert getattr(py, name).offset == off, name


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -1e-3])
def test_non_finite_or_negative_pdf_grid_is_rejected(lib, pdf, bad):
    """gaps_init validates every grid value on the host before any device
    work: a non-finite or negative x f(x, Q^2) is an invalid argument."""
    from paper_2511_19633_gb300 import gaps as G
    g = pdf.copy()
    g[3, 40, 17] = bad
    cfg = G.make_config(2, 13600.0, pdf_grid=g)
    with pytest.raises(G.GapsError) as e:
        G.gaps_init(cfg)
    assert e.value.code == G.GAPS_ERR_INVALID_ARG


@pytest.mark.parametrize("value", [-1, 2_000_000_000])
def test_cycle_cap_out_of_range_is_rejected(lib, pdf, value):
    from paper_2511_19633_gb300 import gaps as G
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf, max_cycles=value)
    with pytest.raises(G.GapsError) as e:
        G.gaps_init(cfg)
    assert e.value.code == G.GAPS_ERR_INVALID_ARG


@pytest.mark.parametrize("precision,schedule,trial_mode", [(1, 2, 0), (1, 1, 2), (1, 1, 3)])
def test_thresholded_grid_needs_a_supported_scheme(lib, precision, schedule, trial_mode):
    """A table with heavy-quark thresholds (the measure correction of App.
    A.2) runs in FP64 and in the mixed-precision kept or redrawn trials of the
    persistent and wavefront schedules; the other combinations are rejected
    before any device work."""
    from paper_2511_19633_gb300 import gaps as G, inputs
    g = inputs.synthetic_pdf_grid(thresholds=True)
    cfg = G.make_config(2, 13600.0, pdf_grid=g, precision=precision, schedule=schedule, trial_mode=trial_mode)
    with pytest.raises(G.GapsError) as e:
        G.gaps_init(cfg)
    assert e.value.code == G.GAPS_ERR_INVALID_ARG


def test_percentile_fit_of_pdf_ratios(lib):
    """gaps_fit_pdf_ratios (host): per transition the nearest-rank 99th and
    99.99th percentiles of the sampled ratios, against numpy."""
    import numpy as np
    from paper_2511_19633_gb300 import gaps as G
    rng = np.random.default_rng(3)
    rows = []
    for num, den, m in ((0, 4, 50000), (11, 0, 20000), (3, 3, 7)):
        r = rng.lognormal(0.0, 1.0, m).astype(np.float32)
        rows.append(np.stack([np.full(m, num), np.full(m, den), rng.uniform(1e-5, 0.9, m), r], 1))
    s = np.concatenate(rows).astype(np.float32)
    fit = G.gaps_fit_pdf_ratios(s)
    for num, den in ((0, 4), (11, 0), (3, 3)):
        r = np.sort(s[(s[:, 0] == num) & (s[:, 1] == den), 3])
        for k, p in ((0, 0.99), (1, 0.9999)):
            assert fit[num, den, k] == r[int(np.ceil(p * r.size)) - 1]
    assert fit[5, 5, 0] == 0.0 and fit[5, 5, 1] == 0.0


def test_percentile_fit_rejects_bad_input(lib):
    import numpy as np
    from paper_2511_19633_gb300 import gaps as G
    for row in ([12, 0, 0.1, 1.0], [0, -1, 0.1, 1.0], [0, 0, 0.1, np.inf]):
        with pytest.raises(Exception):
            G.gaps_fit_pdf_ratios(np.array([row], dtype=np.float32))
    assert np.all(G.gaps_fit_pdf_ratios(np.zeros((0, 4), dtype=np.float32)) == 0.0)
