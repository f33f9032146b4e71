"""CPU checks of the CUDA library: the C ABI loads and exports every declared symbol, and the
host BDD compiler and slab layout reproduce the oracle's canonical BDDs bit for bit."""
from __future__ import annotations

import glob
import os
import re

import numpy as np
import pytest

from instances import SENSE_EQ, SENSE_LE, config, potts_mrf, random_ilp, tomography, tracking
from instances.generators import _from_rows
from oracle import Oracle, OracleError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(bdd_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(cuda_lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(cuda_lib, name), name
    from paper_2009_00481_gb300 import EXPORTED
    assert sorted(EXPORTED) == names


def test_strerror_and_defaults(cuda_lib):
    from paper_2009_00481_gb300 import binding as B
    assert B.bdd_strerror(0) == "ok"
    assert "no 0-1 solution" in B.bdd_strerror(-2)
    opt = B.bdd_default_options()
    assert abs(opt.omega - 0.5) < 1e-7 and opt.host_only == 0 and opt.device == -1


def _lib_canonical(inst, host_only):
    from paper_2009_00481_gb300 import Solver
    s = Solver(inst, host_only=host_only)
    return s, s.canonical()


def _assert_same(inst, host_only):
    o = Oracle(inst)
    want = o.canonical()
    s, got = _lib_canonical(inst, host_only)
    assert (s.nb, s.O, s.N, s.max_depth, s.max_width) == (o.nb, o.O, o.N, o.max_depth, o.max_width)
    for key in ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


@pytest.mark.parametrize("host_only", [1, 2])
@pytest.mark.parametrize("which", ["potts", "matching", "tomography", "tomography_small", "tracking"])
def test_compiler_bit_exact_workloads(cuda_lib, which, host_only):
    """Canonical BDD node and arc arrays equal the oracle's (Prop. 2 canonicity makes the two
    independently built BDDs identical after canonical numbering)."""
    inst = {"potts": lambda: config(0), "matching": lambda: config(1), "tomography": lambda: config(2),
            "tomography_small": lambda: tomography(side=12, seed=3, unary_sigma=0.1),
            "tracking": lambda: tracking(frames=8, dets=30, seed=2)}[which]()
    _assert_same(inst, host_only)


@pytest.mark.parametrize("seed", range(25))
def test_compiler_bit_exact_random(cuda_lib, seed):
    inst = random_ilp(n=30, m=25, max_row_vars=14, seed=700 + seed, coef=3)
    _assert_same(inst, 1 + seed % 2)


@pytest.mark.parametrize("seed", range(20))
def test_compiler_bit_exact_unit_rows(cuda_lib, seed):
    """Rows with coefficients +-1 only (the library compiles them from integer ranges instead of
    sorted sum sets): canonical arrays equal the oracle's for every sense, including rows with
    no feasible completion of some partial sums and one-variable rows."""
    inst = random_ilp(n=40, m=40, max_row_vars=16, seed=900 + seed, coef=1)
    _assert_same(inst, 1 + seed % 2)


def test_compiler_unit_rows_mixed_with_general_rows(cuda_lib):
    """+-1 rows and rows with larger coefficients in one instance, every sense: both paths of
    the compiler, the same canonical arrays as the oracle."""
    rows = [([0, 1, 2, 3], [1, -1, 1, 1], 1, 0), ([1, 2, 4], [2, -3, 1], 0, 1),
            ([0, 3, 4, 5], [-1, -1, 1, 1], 0, -1), ([2, 5], [1, 1], 1, 1), ([5], [-1], -1, 0)]
    inst = _from_rows("mixed", 6, rows, np.random.default_rng(5).normal(size=6))
    for host_only in (1, 2):
        _assert_same(inst, host_only)


def test_layout_classes(cuda_lib):
    """Potts rows have width <= 2 (warp tiles of 16 BDDs); tomography projections are wider than
    32 nodes (one block per BDD)."""
    from paper_2009_00481_gb300 import Solver
    s = Solver(config(0), host_only=2)
    assert s.block_tiles == 0 and s.warp_tiles > 0
    t = Solver(config(2), host_only=2)
    assert t.block_tiles > 0 and t.max_width > 32


def test_build_errors(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300.binding import BDD_EINFEASIBLE, BDD_EINVAL
    dup = _from_rows("dup", 3, [(np.array([1, 1]), np.array([1, 1]), 1, SENSE_LE)], np.zeros(3, np.float32))
    with pytest.raises(BDDError) as e:
        Solver(dup, host_only=1)
    assert e.value.code == BDD_EINVAL
    inf = _from_rows("inf", 3, [(np.array([0, 1]), np.array([1, 1]), 1, SENSE_LE),
                                (np.array([0, 2]), np.array([1, 1]), 3, SENSE_EQ)], np.zeros(3, np.float32))
    with pytest.raises(BDDError) as e:
        Solver(inf, host_only=1)
    assert e.value.code == BDD_EINFEASIBLE and e.value.row == 1
    with pytest.raises(OracleError) as e2:
        Oracle(inf)
    assert e2.value.row == 1
    nan = _from_rows("nan", 1, [(np.array([0]), np.array([1]), 1, SENSE_LE)], np.array([np.nan], np.float32))
    with pytest.raises(BDDError) as e:
        Solver(nan, host_only=1)
    assert e.value.code == BDD_EINVAL
    bad_col = _from_rows("col", 2, [(np.array([0, 5]), np.array([1, 1]), 1, SENSE_LE)], np.zeros(2, np.float32))
    with pytest.raises(BDDError) as e:
        Solver(bad_col, host_only=1)
    assert e.value.code == BDD_EINVAL
    empty = _from_rows("e", 2, [(np.array([], np.int64), np.array([], np.int64), 0, SENSE_LE),
                                (np.array([0, 1]), np.array([0, 1]), 1, SENSE_EQ)], np.zeros(2, np.float32))
    s = Solver(empty, host_only=2)
    assert s.nb == 1 and s.O == 1


def test_host_only_refuses_device_calls(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300.binding import BDD_ESTATE
    s = Solver(potts_mrf(3, 3, 2, seed=0), host_only=1)
    with pytest.raises(BDDError) as e:
        s.iterate(1)
    assert e.value.code == BDD_ESTATE
    with pytest.raises(BDDError) as e:
        s.get_state()
    assert e.value.code == BDD_ESTATE


@pytest.mark.filterwarnings("ignore::DeprecationWarning")
def test_build_in_a_forked_child(cuda_lib):
    """The host compiler's worker threads live in the process that made them: a child forked
    after a build (e.g. a fork-started data-loader worker) compiles on its own thread and does
    not wait for workers it does not have."""
    import os
    import time
    from paper_2009_00481_gb300 import Solver
    inst = config(1)
    Solver(inst, host_only=1)  # the pool exists in this process now
    pid = os.fork()
    if pid == 0:  # child: build again and report
        code = 1
        try:
            s = Solver(inst, host_only=2)
            code = 0 if s.N == Oracle(inst).N else 1
        finally:
            os._exit(code)
    deadline = time.time() + 60
    while True:
        done, status = os.waitpid(pid, os.WNOHANG)
        if done:
            break
        if time.time() > deadline:
            os.kill(pid, 9)
            os.waitpid(pid, 0)
            raise AssertionError("the forked child's build did not finish")
        time.sleep(0.05)
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0


def _tables():
    """Layout tables that move every key to another valid tile class: lane tiles for widths <= 2
    and teams twice as wide above; two-lane teams for widths <= 2 and block tiles for every
    wider key; the defaults."""
    up = [-1] * 28
    blk = [-1] * 28
    for k in range(28):
        c = k // 4
        if c <= 1:
            up[k] = 7
            blk[k] = 1
        elif c < 6:
            up[k] = c + 1
            blk[k] = 6
    return {"lanes_and_wider_teams": up, "teams_and_blocks": blk, "defaults": [-1] * 28}


@pytest.mark.parametrize("which", ["potts", "tomography_small", "tracking", "random"])
@pytest.mark.parametrize("table", sorted(_tables()))
def test_layout_tables_keep_canonical_form(cuda_lib, which, table):
    """Every tile-class table the layout tuner may pick gives slabs whose canonical read-back is
    the oracle's BDDs, bit for bit (host layout, no GPU); the reported table matches."""
    from paper_2009_00481_gb300 import Solver
    inst = {"potts": lambda: config(0), "tomography_small": lambda: tomography(side=12, seed=3, unary_sigma=0.1),
            "tracking": lambda: tracking(frames=8, dets=30, seed=2),
            "random": lambda: random_ilp(n=40, m=30, max_row_vars=14, seed=5, coef=3)}[which]()
    tab = np.asarray(_tables()[table], np.int32)
    s = Solver(inst, host_only=2, layout_classes=tab)
    want = Oracle(inst).canonical()
    got = s.canonical()
    for key in ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
    rep = s.layout_table()
    assert rep["nodes"].sum() == s.N
    for k in range(28):
        if rep["nodes"][k] == 0:
            assert rep["cls"][k] == -1
        elif tab[k] >= 0:
            assert rep["cls"][k] == tab[k]
    assert s.lanes == int(table == "lanes_and_wider_teams")


def test_layout_table_rejects_narrow_classes(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300.binding import BDD_EINVAL
    inst = tomography(side=12, seed=3, unary_sigma=0.1)
    bad = np.full(28, -1, np.int32)
    bad[3 * 4: 4 * 4] = 2  # widths 5..8 in teams of 4 lanes
    with pytest.raises(BDDError) as e:
        Solver(inst, host_only=2, layout_classes=bad)
    assert e.value.code == BDD_EINVAL
    lanes_wide = np.full(28, -1, np.int32)
    lanes_wide[8:12] = 7  # lane tiles are for widths <= 2 only
    with pytest.raises(BDDError) as e:
        Solver(inst, host_only=2, layout_classes=lanes_wide)
    assert e.value.code == BDD_EINVAL
    with pytest.raises(BDDError) as e:  # explicit tables are for plain solvers
        Solver(inst, host_only=2, layout_classes=np.full(28, -1, np.int32), alpha=0.1)
    assert e.value.code == BDD_EINVAL


def test_device_error_word_mapping(cuda_lib):
    """A device error word maps to a status on the host: 0 ok, -7 (an index check of the checked
    build failed) BDD_EDEVICE, anything else (a bounded device-side wait gave up) BDD_ETIMEOUT."""
    from paper_2009_00481_gb300.binding import BDD_EDEVICE, BDD_ETIMEOUT, BDD_OK
    f = cuda_lib.bdd_status_of_device_word
    assert f(0) == BDD_OK
    assert f(-7) == BDD_EDEVICE
    assert f(-6) == BDD_ETIMEOUT and f(1) == BDD_ETIMEOUT and f(-1) == BDD_ETIMEOUT


def test_checked_library_exports_the_same_symbols(cuda_lib):
    """The checked build (-DBDD_CHECKED sweep kernels) loads without a GPU and exports the same
    C ABI; BDD_DBCA_CHECKED=1 selects it as the process's library."""
    import ctypes
    from paper_2009_00481_gb300 import binding
    from paper_2009_00481_gb300.build import LIB_CHECKED
    lib = ctypes.CDLL(LIB_CHECKED)
    for name in declared_functions():
        assert hasattr(lib, name), name
    old = os.environ.get("BDD_DBCA_CHECKED")
    try:
        os.environ["BDD_DBCA_CHECKED"] = "1"
        assert binding.default_library() == LIB_CHECKED
        os.environ["BDD_DBCA_CHECKED"] = "0"
        assert binding.default_library() == binding.LIB
    finally:
        if old is None:
            os.environ.pop("BDD_DBCA_CHECKED", None)
        else:
            os.environ["BDD_DBCA_CHECKED"] = old
