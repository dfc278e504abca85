"""Host logic of the CUDA path, on the CPU: the explicit operator rows the
builder derives (used by the sparse-row kernels and the adjoints), its
least-squares class tables as the interpolation kernel applies them, and
its restriction rows, compared with the oracle's rows for the finite-
difference and least-squares schemes, patch sizes that are and are not
multiples of 3.  A small harness (tests/host/builder_rows.cpp) is compiled
against the builder sources with the CUDA toolkit's nvcc."""
import collections
import os
import shutil
import subprocess

import pytest

from oracle import operators as op

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("host") / "builder_rows")
    cmd = [nvcc, "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "host", "builder_rows.cpp"),
           os.path.join(ROOT, "paper_2504_15814_gb300", "csrc", "builder.cpp")]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def _rows(exe, *args):
    out = subprocess.run([exe, *map(str, args)], check=True, capture_output=True, text=True).stdout
    rows = collections.defaultdict(dict)
    for line in out.splitlines():
        o, c, w = line.split()
        rows[int(o)][int(c)] = rows[int(o)].get(int(c), 0.0) + float(w)
    return rows


def _worst(got, outs, rows):
    assert set(got) <= set(outs)
    worst = 0.0
    for o, row in zip(outs, rows):
        g = got.get(o, {})
        scale = max(1.0, max(abs(w) for w in row.values()))
        worst = max(worst, max(abs(g.get(c, 0.0) - row.get(c, 0.0)) for c in set(g) | set(row)) / scale)
    return worst


CASES = [(9, 3, 3, 4), (9, 3, 2, 0), (6, 2, 3, 8), (8, 3, 3, 2), (5, 2, 2, 4), (4, 3, 3, 6), (12, 2, 3, 1)]


DLINEAR = [(9, 3, 1, 4), (7, 2, 1, 3), (5, 1, 1, 0)]


@pytest.mark.parametrize("p,k,order,sub", CASES + DLINEAR)
@pytest.mark.parametrize("scheme", [op.SCHEME_FD, op.SCHEME_LS])
def test_interpolation_rows_match_oracle(harness, p, k, order, sub, scheme):
    if order == 1 and scheme == op.SCHEME_LS:
        pytest.skip("least squares needs a Taylor order")
    outs, rows = op.interpolation_rows(0, sub, p, k, order, scheme=scheme)
    assert _worst(_rows(harness, "interp", p, k, order, sub, scheme), outs, rows) < 1e-13


@pytest.mark.parametrize("p,k,order,sub", CASES + DLINEAR)
@pytest.mark.parametrize("scheme", [op.SCHEME_FD, op.SCHEME_LS])
def test_restriction_rows_match_oracle(harness, p, k, order, sub, scheme):
    if order == 1 and scheme == op.SCHEME_LS:
        pytest.skip("least squares needs a Taylor order")
    outs, rows = op.restriction_rows(0, sub, p, k, order, scheme=scheme)
    assert _worst(_rows(harness, "restrict", p, k, order, sub, scheme), outs, rows) < 1e-13


@pytest.mark.parametrize("p,k,order,sub", CASES)
def test_least_squares_class_tables_match_oracle(harness, p, k, order, sub):
    """The per-class fit tables, applied over the kernel's stencil slots,
    give the oracle's least-squares interpolation rows."""
    outs, rows = op.interpolation_rows(0, sub, p, k, order, scheme=op.SCHEME_LS)
    assert _worst(_rows(harness, "lsclass", p, k, order, sub), outs, rows) < 1e-13


@pytest.mark.parametrize("p,k,order,sub", [(9, 3, 3, -1), (12, 3, 3, -1), (6, 2, 2, -1), (16, 3, 3, 4), (24, 3, 1, -1),
                                           (48, 3, 3, -1), (7, 3, 3, -1), (4, 2, 3, 0), (9, 1, 1, -1),
                                           (9, 4, 3, -1), (9, 5, 3, 4), (12, 5, 2, -1), (9, 4, 1, -1), (9, 5, 1, 7)])
@pytest.mark.parametrize("budget", [64 * 1024, 112 * 1024])
def test_fixed_point_tiles_fit_their_launch(harness, p, k, order, sub, budget):
    """Fixed-point plans (precision 2): every tile of the fixed-point kernel
    carries at most 32 unknowns and its region, at 32 slots of 8 bytes per
    volume, fits the shared memory the launch provides (and the budget,
    unless a single centre's region exceeds it); the tiles cover every
    coarse centre of the item once per unknown."""
    U = 59
    out = subprocess.run([harness, "tiles", *map(str, (p, k, order, sub, 2, U, budget))], check=True, capture_output=True,
                         text=True).stdout.split("\n")
    smem = int([line for line in out if line.startswith("smem")][0].split()[1])
    cover = collections.Counter()
    for line in out:
        if not line or line.startswith("smem"):
            continue
        seg, a0, na, b0, nb, u0, nu, vols = map(int, line.split())
        assert seg in (0, 1) and 1 <= nu <= 32
        assert vols * 32 * 8 <= smem <= 227 * 1024
        if na * nb > 1:
            assert vols * 32 * 8 <= budget
        for a in range(a0, a0 + na):
            for b in range(b0, b0 + nb):
                for u in range(u0, u0 + nu):
                    cover[(a, b, u)] += 1
    if sub < 0:
        lo_a, hi_a, lo_b, hi_b = 0, p, 0, p
    else:
        s0, s1 = sub % 3, sub // 3
        lo_a, hi_a = (s0 * p) // 3, (s0 * p + p - 1) // 3 + 1
        lo_b, hi_b = (s1 * p) // 3, (s1 * p + p - 1) // 3 + 1
    assert set(cover.values()) == {1}
    assert len(cover) == (hi_a - lo_a) * (hi_b - lo_b) * U
