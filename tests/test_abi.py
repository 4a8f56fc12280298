"""The C-ABI library builds, loads without a GPU, exports every function the
header declares, and validates its arguments before touching the GPU."""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_18889_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2411_18889_gb300 import build
        build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_2411_18889_gb300 import _lib
    names = _lib.header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), f"{name} declared in nbody.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_batched_shape_count(lib):
    """The GPU tests run every batched shape; they assume six (the build's
    instantiations)."""
    from paper_2411_18889_gb300 import build
    assert lib.nbody_num_batched_configs() == build.NUM_BATCHED_SHAPES == 6


def test_static_queries(lib):
    assert lib.nbody_version() >= 10000
    k = lib.nbody_num_configs()
    assert k >= 1
    for i in range(k):
        b = lib.nbody_config_block(i)
        assert b > 0 and b % 64 == 0
    assert lib.nbody_config_block(-1) == 0 and lib.nbody_config_block(k) == 0
    assert lib.nbody_strerror(0) == b"success"
    assert lib.nbody_strerror(-1) == b"invalid argument"
    assert lib.nbody_strerror(-4) == b"bounded device wait expired"


def test_argument_validation_without_gpu(lib):
    from paper_2411_18889_gb300._lib import NBODY_EINVAL, NBODY_OK, NbodyOpts
    p = np.zeros((4, 3))
    pf = np.zeros((4, 3), dtype=np.float32)
    m = np.ones(4, dtype=np.float32)
    a = np.zeros((4, 3), dtype=np.float32)
    vp = lambda x: ctypes.c_void_p(x.ctypes.data)
    nul = None
    # n == 0 is a no-op
    assert lib.nbody_accel(0, nul, nul, 0.1, nul, nul, nul) == NBODY_OK
    assert lib.nbody_leapfrog(0, nul, nul, nul, 0.1, 0.01, 5, nul) == NBODY_OK
    assert lib.nbody_leapfrog_f32(4, vp(pf), vp(pf), vp(m), 0.1, 0.01, 0, nul) == NBODY_OK  # zero steps
    # bad sizes, pointers, softening, time step
    assert lib.nbody_accel(-1, vp(p), vp(m), 0.1, vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel(4, nul, vp(m), 0.1, vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel(4, vp(p), nul, 0.1, vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel(4, vp(p), vp(m), 0.1, nul, nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel(4, vp(p), vp(m), -0.1, vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel(4, vp(p), vp(m), float("nan"), vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_accel_f32(4, vp(pf), vp(m), float("inf"), vp(a), nul, nul) == NBODY_EINVAL
    assert lib.nbody_leapfrog(4, vp(p), vp(p), vp(m), 0.1, float("nan"), 1, nul) == NBODY_EINVAL
    assert lib.nbody_leapfrog(4, vp(p), vp(p), vp(m), 0.1, 0.01, -1, nul) == NBODY_EINVAL
    assert lib.nbody_leapfrog_f32(4, vp(pf), nul, vp(m), 0.1, 0.01, 1, nul) == NBODY_EINVAL
    out = np.zeros(9)
    assert lib.nbody_energy(4, vp(p), vp(p), vp(m), 0.1, nul, nul) == NBODY_EINVAL
    assert lib.nbody_energy(0, nul, nul, nul, 0.1, vp(out), nul) == NBODY_OK
    # options
    o = NbodyOpts()
    lib.nbody_opts_default(ctypes.byref(o))
    assert (o.precision, o.accumulate, o.config, o.reserved) == (0, 0, -1, 0)
    for field, bad in (("precision", 7), ("accumulate", 3), ("config", 999), ("config", -2), ("reserved", 1)):
        o2 = NbodyOpts()
        lib.nbody_opts_default(ctypes.byref(o2))
        setattr(o2, field, bad)
        assert lib.nbody_accel(4, vp(p), vp(m), 0.1, vp(a), nul, ctypes.byref(o2)) == NBODY_EINVAL


def test_python_binding_checks_arrays():
    import paper_2411_18889_gb300 as nb
    p = np.zeros((4, 3), dtype=np.float32)  # wrong dtype for nbody_accel
    m = np.ones(4, dtype=np.float32)
    a = np.zeros((4, 3), dtype=np.float32)
    with pytest.raises(TypeError):
        nb.nbody_accel(p, m, 0.1, a)
    with pytest.raises(ValueError):
        nb.nbody_accel_f32(p, m[:3], 0.1, a)
    with pytest.raises(ValueError):
        nb.nbody_accel_f32(np.zeros((3, 4), dtype=np.float32).T, m[:3], 0.1, a)


def test_tune_table_parse_and_query(lib, tmp_path):
    """The shape table: built-in rules, a file's rules (largest n_min <= n wins),
    rejection of malformed lines and out-of-range shapes (table unchanged)."""
    EINVAL = -1
    good = tmp_path / "t.txt"
    good.write_text("# comment\nforce 0 0 3\nforce 0 5000 2\nforce 1 0 0\nvjp 0 1\nvjp 100000 2\nbatched 3\n"
                    "batched 1024 0\n")
    assert lib.nbody_tune_load(str(good).encode()) == 7
    assert lib.nbody_tuned_shape(0, 10, 0) == 3
    assert lib.nbody_tuned_shape(0, 5000, 0) == 2
    assert lib.nbody_tuned_shape(0, 10 ** 7, 1) == 0
    assert lib.nbody_tuned_shape(1, 99999, 0) == 1
    assert lib.nbody_tuned_shape(1, 100000, 0) == 2
    assert lib.nbody_tuned_shape(2, 1023, 0) == 3  # batched rules key on the largest system
    assert lib.nbody_tuned_shape(2, 4096, 0) == 0
    for bad in ("force 0 0 99\n", "force 2 0 1\n", "vjp -5 1\n", "nonsense 1 2\n", "force 0\n", "batched 0 9\n",
                "batched -1 0\n"):
        f = tmp_path / "bad.txt"
        f.write_text(bad)
        assert lib.nbody_tune_load(str(f).encode()) == EINVAL
        assert lib.nbody_tuned_shape(0, 5000, 0) == 2  # unchanged
    assert lib.nbody_tune_load(str(tmp_path / "missing.txt").encode()) == EINVAL
    assert lib.nbody_tuned_shape(3, 10, 0) == EINVAL
    assert lib.nbody_tune_load(None) >= 0  # back to the default location / built-in table
    for n in (1, 1000, 1 << 20):
        for pot in (0, 1):
            assert 0 <= lib.nbody_tuned_shape(0, n, pot) < lib.nbody_num_configs()


def test_tune_table_batched_shapes(lib, tmp_path):
    """Batched rules are checked against the batched shapes (six), not the
    force shapes (five): the last batched shape loads, one past it does not."""
    k = lib.nbody_num_batched_configs()
    f = tmp_path / "b.txt"
    f.write_text(f"force 0 0 3\nbatched 0 {k - 1}\n")
    assert lib.nbody_tune_load(str(f).encode()) == 2
    assert lib.nbody_tuned_shape(2, 4096, 0) == k - 1
    f.write_text(f"force 0 0 3\nbatched 0 {k}\n")
    assert lib.nbody_tune_load(str(f).encode()) == -1
    assert lib.nbody_tuned_shape(2, 4096, 0) == k - 1  # unchanged
    assert lib.nbody_tune_load(None) >= 0


def test_tune_table_fault_injection(lib, tmp_path, monkeypatch):
    """NBODY_FAULT=tune: reading a shape table fails as if the file were bad;
    the built-in table keeps serving and nothing touches a GPU."""
    good = tmp_path / "t.txt"
    good.write_text("force 0 0 3\nvjp 0 1\nbatched 3\n")
    monkeypatch.setenv("NBODY_FAULT", "tune")
    assert lib.nbody_tune_load(str(good).encode()) == -1
    assert lib.nbody_tune_load(None) == 0  # default location unreadable: built-in table
    for n in (1, 1000, 1 << 20):
        assert 0 <= lib.nbody_tuned_shape(0, n, 0) < lib.nbody_num_configs()
    monkeypatch.delenv("NBODY_FAULT")
    assert lib.nbody_tune_load(str(good).encode()) == 3
    assert lib.nbody_tuned_shape(0, 10, 0) == 3
    assert lib.nbody_tune_load(None) >= 0


def test_tuner_rules_round_trip(lib, tmp_path):
    """The survey's size ladder becomes rules that start each winner at the
    midpoint below its size and merge repeats; written in the table format,
    the library reads them back and answers with the same winners."""
    from paper_2411_18889_gb300.tune import _rules
    sizes = [1024, 4096, 16384, 32768, 65536]
    winners = [4, 4, 3, 2, 2]
    rules = _rules(sizes, winners)
    assert rules == [(0, 4), (10240, 3), (24576, 2)]
    f = tmp_path / "t.txt"
    f.write_text("".join(f"force 0 {a} {k}\n" for a, k in rules) + "".join(f"batched {a} {min(k, 3)}\n" for a, k in rules))
    assert lib.nbody_tune_load(str(f).encode()) == 2 * len(rules)
    for n, k in zip(sizes, winners):
        assert lib.nbody_tuned_shape(0, n, 0) == k
        assert lib.nbody_tuned_shape(2, n, 0) == min(k, 3)
    assert lib.nbody_tune_load(None) >= 0


def test_product_path_does_not_use_the_oracle():
    """The package and its CUDA sources never import, load or name the oracle
    (it is test infrastructure), and loading fails loudly without the built
    library instead of falling back to anything."""
    import glob
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2411_18889_gb300")
    files = glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*"))
    assert files
    for f in files:
        src = open(f, errors="replace").read()
        assert not re.search(r"\boracle\b", src), f
    from paper_2411_18889_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.open_library(os.path.join(pkg, "no_such_libnbody.so"))
