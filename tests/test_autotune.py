"""The tuned-table option (host side): a table written in the autotuner's
format sets the cut-overs of the first matching size class at analysis."""
import os

import pytest

from paper_2510_05885_gb300 import ncl_kkt as nk
from paper_2510_05885_gb300 import synth


def _write(tmp_path, text):
    p = tmp_path / "tuned.txt"
    p.write_text(text)
    return str(p)


def _handle(form, side, **opts):
    pat = synth.make_pattern(side, side)
    return nk.KKT(form, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, host_only=1, **opts)


def test_first_matching_line_sets_the_cutovers(tmp_path):
    path = _write(tmp_path, "# comment\n"
                            "1 0 100 1 1 1 1 2 64   # too small a range for the test system\n"
                            "0 0 100000 1 1 0 0 1 128  # the stabilized 12 x 12 grid (dim 864)\n"
                            "0 0 100000 1 1 1 1 2 512  # not reached: the line above matches first\n")
    K = _handle(0, 12, autotune_path=path)
    o = nk.ncl_kkt_get_options(K._h)
    assert (o.persistent_fronts, o.subtree_sweeps, o.use_tensor_cores, o.tc_min_pivots) == (0, 0, 1, 128)
    assert o.autotune_path is None
    K.close()


def test_no_matching_line_keeps_the_defaults(tmp_path):
    path = _write(tmp_path, "1 0 1000000 1 1 0 0 0 64\n")
    K = _handle(0, 12, autotune_path=path)
    o = nk.ncl_kkt_get_options(K._h)
    d = nk.default_options()
    assert (o.persistent_fronts, o.subtree_sweeps, o.use_tensor_cores, o.tc_min_pivots) == \
        (d.persistent_fronts, d.subtree_sweeps, d.use_tensor_cores, d.tc_min_pivots)
    K.close()


def test_batch_count_ranges(tmp_path):
    path = _write(tmp_path, "0 0 1000000 1 1 1 1 2 256\n0 0 1000000 2 8 0 1 2 512\n")
    pats = [synth.make_pattern(6, 7) for _ in range(3)]
    K = nk.KKT.batch(0, [(p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind) for p in pats], host_only=1,
                     autotune_path=path)
    o = nk.ncl_kkt_get_options(K._h)
    assert (o.persistent_fronts, o.tc_min_pivots) == (0, 512)
    K.close()


@pytest.mark.parametrize("text", ["0 0 100\n", "0 0 100000 1 1 2 0 2 256\n", "0 0 100000 1 1 1 1 2 16\n"])
def test_bad_lines_are_refused(tmp_path, text):
    path = _write(tmp_path, text)
    with pytest.raises(nk.NclError) as e:
        _handle(0, 6, autotune_path=path)
    assert e.value.status == 1 and "tuned table" in str(e.value)


def test_missing_table_is_refused(tmp_path):
    with pytest.raises(nk.NclError) as e:
        _handle(0, 6, autotune_path=os.path.join(str(tmp_path), "absent.txt"))
    assert e.value.status == 1


def test_tensor_core_threshold_is_validated():
    with pytest.raises(nk.NclError):
        _handle(0, 6, tc_min_pivots=8)


def test_committed_table_parses():
    """The table the autotuner wrote on the GB300 is accepted as it stands."""
    from paper_2510_05885_gb300 import autotune
    path = os.path.join(os.path.dirname(autotune.__file__), "tuned_gb300.txt")
    if not os.path.exists(path):
        pytest.skip("no tuned table committed")
    K = _handle(1, 20, autotune_path=path)
    assert nk.ncl_kkt_get_options(K._h).tc_min_pivots >= 32
    K.close()


@pytest.mark.parametrize("mode", [-1, 3])
def test_precision_fallback_mode_is_validated(mode):
    with pytest.raises(nk.NclError):
        _handle(0, 6, precision_fallback=mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_precision_fallback_modes_accepted(mode):
    K = _handle(1, 6, precision_fallback=mode)
    assert nk.ncl_kkt_get_options(K._h).precision_fallback == mode
    K.close()


def _table_lines(path):
    out = []
    for ln in open(path):
        body = ln.split("#", 1)[0].split()
        if body:
            out.append([int(v) for v in body])
    return out


def test_committed_table_classes_are_disjoint():
    """No two lines of the committed table can match the same analysis, so
    the first-match rule never hides a line."""
    from paper_2510_05885_gb300 import autotune
    path = os.path.join(os.path.dirname(autotune.__file__), "tuned_gb300.txt")
    lines = _table_lines(path)
    assert len(lines) >= 6
    for i, a in enumerate(lines):
        assert len(a) == 9 and a[1] < a[2] and a[3] <= a[4]
        for b in lines[i + 1:]:
            same_form = a[0] == b[0]
            dims = a[1] < b[2] and b[1] < a[2]
            counts = a[3] <= b[4] and b[3] <= a[4]
            assert not (same_form and dims and counts), (a, b)


@pytest.mark.parametrize("form,R,C,want", [
    (0, 20, 25, (0, 0, 128)),     # the 20 x 25 workload: the tiny stabilized class
    (1, 300, 300, (0, 0, 128)),   # the default workload: the condensed 300 x 300 class
])
def test_benchmark_workloads_get_their_class(form, R, C, want):
    from paper_2510_05885_gb300 import autotune
    path = os.path.join(os.path.dirname(autotune.__file__), "tuned_gb300.txt")
    pat = synth.make_pattern(R, C)
    K = nk.KKT(form, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, host_only=1,
               autotune_path=path)
    o = nk.ncl_kkt_get_options(K._h)
    assert (o.persistent_fronts, o.subtree_sweeps, o.tc_min_pivots) == want
    K.close()
