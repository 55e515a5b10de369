"""Cut cells that fill several chunks of the cut-cell kernel, against the FP64 oracle.

The cut-cell kernel hands each cut cell to a group of S lanes (S = 32, 16 or 8; the FP32 kernel
runs the 16-lane class with 32 lanes) and walks the cell's volume lines axis by axis in chunks of
at most S lines, one line per lane.  The lines of an axis come in groups that share one outer
coordinate; a chunk holds at most GMAX groups (16 for n <= 5, 8 for n = 6..8, 6 for n = 9, and never more than S / 2
in the 16- and 8-lane classes) and ends before the start of group GMAX + 1, and a group that does
not fit restarts in the next chunk.  `chunks_of_cell` restates that rule from the exported line structure, so that the tests
can assert which paths their cells take:
  * an axis whose lines need more than one chunk;
  * a chunk ended early because it reached GMAX groups;
  * a group cut by a chunk boundary (its lines in two chunks);
  * cells with more than 1,000 volume points (the paper's Sec. 6.1 notes cut cells with over
    1,000 points in its many-sphere geometries).
The rows of those cells are compared element by element with the oracle (FP64 1e-12, FP32 1e-5
against the oracle on the FP32-rounded input, adjoint 1e-12), on small unions of balls and on the
largest cells of the random 100-spheres Q3 workload at full size.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import forms, mesh

TOL64 = 1e-12
TOL32 = 1e-5


def cut_gmax(n):
    return 16 if n <= 5 else 8 if n <= 8 else 6


def chunks_of_cell(axis, group_start, lanes, n):
    """Chunks of the 3D volume phase of one cut cell: (axis, first line within the axis, lines,
    ended because it reached GMAX groups, a group continues in the next chunk)."""
    gmax = min(cut_gmax(n), lanes if lanes >= 32 else lanes // 2)
    out = []
    for k in range(3):
        idx = np.nonzero(axis == k)[0]
        if len(idx) == 0:
            continue
        lb, le = int(idx[0]), int(idx[-1]) + 1
        l0 = lb
        while l0 < le:
            cand = range(l0, min(l0 + lanes, le))
            starts = [t for t in cand if t == l0 or group_start[t]]
            if len(starts) > gmax:
                nl, by_gmax = starts[gmax] - l0, True
            else:
                nl, by_gmax = len(cand), False
            cut_group = (l0 + nl < le) and not group_start[l0 + nl]
            out.append((k, l0 - lb, nl, by_gmax, cut_group))
            l0 += nl
    return out


def chunk_features(op, c, lanes64, n):
    """{precision: set of features} of cut cell c: 'multi' (an axis in several chunks), 'gmax',
    'group_cut'."""
    axis, gs, _ = op.export_cut_cell_lines(c)
    feats = {}
    for prec, lanes in (("fp64", lanes64), ("fp32", 32 if lanes64 == 16 else lanes64)):
        ch = chunks_of_cell(axis, gs, lanes, n)
        per_axis = np.bincount([k for k, *_ in ch], minlength=3)
        f = set()
        if per_axis.max() > 1:
            f.add("multi")
        if any(x[3] for x in ch):
            f.add("gmax")
        if any(x[4] for x in ch):
            f.add("group_cut")
        feats[prec] = f
    return feats


# unions of intersecting balls whose cells carry many lines: n = 4 (GMAX 16, the headline
# kernel's instance) with 6 Gauss points per interval, n = 7 (GMAX 8), and n = 3 with its 16- and
# 32-lane classes
CASES = {
    "3d_random_spheres_q3_6_q6": dict(workloads.spheres_random(p=3, N=6, n=10, R=(0.1, 0.3), seed=3),
                                      quad_order=6),
    "3d_random_spheres_q6_4": workloads.spheres_random(p=6, N=4, n=10, R=(0.1, 0.3), seed=3),
    "3d_random_spheres_q2_10": workloads.spheres_random(p=2, N=10, n=8, R=0.22, seed=5),
}


def _host_op(cfg):
    from paper_2404_07911_gb300 import UnfittedOperator

    return UnfittedOperator(cfg, device=-1)


def select_cells(op, n, per_feature=3):
    """Cut cells (cut-cell index) covering every chunk feature in both precisions, plus the cells
    with the most lines; returns (selection, {(precision, feature): count over all cut cells})."""
    vp, vl, fl, lanes = op.export_cut_cell_counts()
    found = {}
    chosen = []
    for c in np.argsort(-vl, kind="stable"):
        c = int(c)
        feats = chunk_features(op, c, int(lanes[c]), n)
        take = False
        for prec, fs in feats.items():
            for f in fs:
                found[(prec, f)] = found.get((prec, f), 0) + 1
                take |= found[(prec, f)] <= per_feature
        if take or len(chosen) < 2:
            chosen.append(c)
    return sorted(set(chosen)), found, vp


@pytest.mark.parametrize("key", list(CASES))
def test_chunk_model_covers_every_path(key):
    """Host only: the selected cells of each case take every chunk path in both precisions."""
    cfg = CASES[key]
    op = _host_op(cfg)
    cells, found, vp = select_cells(op, cfg["degree"] + 1)
    for prec in ("fp64", "fp32"):
        for f in ("multi", "gmax", "group_cut"):
            assert found.get((prec, f), 0) > 0, (key, prec, f)
    assert vp[cells].max() > 1000
    op.close()


def test_chunk_model_on_a_single_group_axis():
    """The rule itself: 40 lines of one axis in groups of 6 on 32 lanes with GMAX 16 take two
    chunks, the first ending inside the sixth group; 40 one-line groups reach GMAX after 16
    lines."""
    axis = np.zeros(40, dtype=np.int32)
    gs = np.zeros(40, dtype=np.int32)
    gs[::6] = 1
    ch = chunks_of_cell(axis, gs, 32, 4)
    assert [(x[1], x[2]) for x in ch] == [(0, 32), (32, 8)]
    assert ch[0][4] and not ch[0][3]
    gs[:] = 1
    ch = chunks_of_cell(axis, gs, 32, 4)
    assert [(x[1], x[2], x[3]) for x in ch] == [(0, 16, True), (16, 16, True), (32, 8, False)]
    ch = chunks_of_cell(axis, gs, 32, 7)  # GMAX 8
    assert [x[2] for x in ch] == [8] * 5


# ----------------------------------------------------------------------------------- GPU rows
def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _rows(op, x, cells, dtype, adjoint=False):
    import torch

    nd = op.info["dofs_per_cell"]
    xt = torch.from_numpy(np.asarray(x)).to(device="cuda", dtype=dtype)
    y = op.vmult_adjoint(xt) if adjoint else op.vmult(xt)
    torch.cuda.synchronize()
    return y.double().cpu().numpy().reshape(-1, nd)[cells]


def _compare_rows(cfg, op, o, cut_sel):
    cut_active = np.nonzero(o.mesh.active_type == mesh.CUT)[0]
    cells = [int(cut_active[c]) for c in cut_sel]
    import torch

    x = workloads.uniform_vector(op.n_dofs, cfg["seed"])
    ref = o.apply_rows(x, cells)
    assert _rel(_rows(op, x, cells, torch.float64), ref) <= TOL64
    assert _rel(_rows(op, x, cells, torch.float64, adjoint=True), o.apply_rows(x, cells, transpose=True)) <= TOL64
    x32 = x.astype(np.float32).astype(np.float64)
    assert _rel(_rows(op, x32, cells, torch.float32), o.apply_rows(x32, cells)) <= TOL32


@pytest.mark.gpu
@pytest.mark.parametrize("key", list(CASES))
def test_rows_of_multichunk_cells(key):
    pytest.importorskip("torch")
    from paper_2404_07911_gb300 import UnfittedOperator

    cfg = CASES[key]
    host = _host_op(cfg)
    cut_sel, found, vp = select_cells(host, cfg["degree"] + 1)
    host.close()
    op = UnfittedOperator(cfg, device=0)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    _compare_rows(cfg, op, o, cut_sel)
    op.close()


@pytest.mark.gpu
def test_random_spheres_q3_largest_cells():
    """The random 100-spheres Q3 workload at full size (192^3 background cells): the cut cells
    with the most volume lines, all above 1,000 points, against the oracle's rows."""
    torch = pytest.importorskip("torch")
    from paper_2404_07911_gb300 import UnfittedOperator

    cfg = workloads.cfg_spheres_random(p=3)
    op = UnfittedOperator(cfg, device=0)
    vp, vl, fl, lanes = op.export_cut_cell_counts()
    biggest = [int(c) for c in np.argsort(-vl, kind="stable")[:6]]
    assert vp[biggest].min() > 1000
    for c in biggest:
        feats = chunk_features(op, c, int(lanes[c]), cfg["degree"] + 1)
        assert "multi" in feats["fp64"] and "multi" in feats["fp32"]
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    _compare_rows(cfg, op, o, biggest)
    op.close()
    torch.cuda.empty_cache()


@pytest.mark.gpu
def test_vmult_refuses_overlapping_vectors():
    """x and y of uf_vmult / uf_vmult_adjoint must not overlap: UF_EINVAL before any launch."""
    torch = pytest.importorskip("torch")
    from paper_2404_07911_gb300 import UnfittedOperator, binding

    lib = binding.load_library()
    op = UnfittedOperator(workloads.small(p=2, N=6), device=0)
    n = op.n_dofs
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for dtype, prec in ((torch.float64, binding.UF_FP64), (torch.float32, binding.UF_FP32)):
        buf = torch.zeros(2 * n + 1, dtype=dtype, device="cuda")
        x = buf[:n]
        esz = buf.element_size()
        for fn in (lib.uf_vmult, lib.uf_vmult_adjoint):
            for shift in (0, 1, n - 1):
                y_ptr = ctypes.c_void_p(x.data_ptr() + shift * esz)
                assert fn(op._h, prec, y_ptr, ctypes.c_void_p(x.data_ptr()), stream) == binding.UF_EINVAL
                assert b"overlap" in lib.uf_last_error()
            # disjoint halves of the same buffer are accepted
            y_ptr = ctypes.c_void_p(x.data_ptr() + n * esz)
            assert fn(op._h, prec, y_ptr, ctypes.c_void_p(x.data_ptr()), stream) == binding.UF_OK
    torch.cuda.synchronize()
    op.close()
