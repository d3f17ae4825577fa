"""The C-ABI library builds, loads without a GPU and exports every entry point of include/xdg.h."""
import ctypes
import os
import re

from paper_2003_02431_gb300 import xdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(xdg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("xdg_create_hierarchy", "xdg_apply", "xdg_vcycle", "xdg_solve", "xdg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    xdg.build()
    lib = ctypes.CDLL(xdg.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in xdg.SIGNATURES}
    assert set(_declared()) <= bound


def test_strerror_without_gpu():
    lib = xdg.load()
    assert lib.xdg_strerror(0) == b"XDG_OK"
    assert lib.xdg_strerror(4) == b"XDG_ENOTCONV"


def _batch_rc(problems):
    import ctypes as C
    keep = []
    arr = (xdg.Problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = xdg._marshal(p.Np, p.nb, p.row_ptr, p.col, p.val, p.agg, p.R, keep)
    h = C.c_void_p()
    lib = xdg.load()
    rc = lib.xdg_create_batch(len(problems), arr, None, None, C.byref(h))
    return rc, lib.xdg_last_error().decode()


def test_batch_validation_names_the_problem_without_gpu():
    """Every index of every batch member is checked on the host before any CUDA call."""
    import numpy as np
    import xdg_problem as xp
    cfgs = xp.batch_configs(4, seed=5, N_range=(8, 12), ks=(2,), max_levels=3)
    probs = [xp.Problem(c) for c in cfgs]

    class P:  # a mutable copy of a problem's arrays
        def __init__(self, p):
            self.Np, self.nb = p.Np, list(p.nb)
            self.row_ptr, self.col, self.val = p.row_ptr.copy(), p.col.copy(), p.val.copy()
            self.agg, self.R = [a.copy() for a in p.agg], [r.copy() for r in p.R]

    cases = []
    bad = P(probs[2])
    bad.agg[1][0] = bad.nb[2]  # coarse index out of range on level 2
    cases.append((2, bad, "agg"))
    bad = P(probs[1])
    bad.col[0] = bad.nb[0]  # column index out of range
    cases.append((1, bad, "col"))
    bad = P(probs[3])
    r = int(np.argmax(np.diff(bad.row_ptr) > 1))
    z = int(bad.row_ptr[r])
    bad.col[z], bad.col[z + 1] = bad.col[z + 1], bad.col[z]  # columns not increasing
    cases.append((3, bad, "increasing"))
    for idx, broken, word in cases:
        lst = [P(p) for p in probs]
        lst[idx] = broken
        rc, msg = _batch_rc(lst)
        assert rc == xdg.XDG_EINVAL, (idx, msg)
        assert ("problem %d" % idx) in msg and word in msg, msg


def test_batch_rejects_unsupported_block_sizes_without_gpu():
    """Batches take the block sizes of the low-precision cycle (6, 10, 15, 20): another Np is
    refused on the host, naming the problem, before any CUDA call."""
    import xdg_problem as xp
    ok = xp.Problem(xp.batch_configs(1, seed=5, N_range=(8, 8), ks=(2,), max_levels=3)[0])
    wide = xp.Problem(xp.Config(D=3, N=2, k=5, c=(0.5, 0.5, 0.5), R=0.3, max_levels=1))
    assert wide.Np == 56
    rc, msg = _batch_rc([ok, wide])
    assert rc == xdg.XDG_EINVAL and "problem 1" in msg and "Np = 56" in msg, msg


def test_binding_argument_counts_match_prototypes():
    """Every ctypes signature has as many arguments as the header's prototype."""
    protos = {}
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, fn)).read(), flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(xdg_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.M):
                args = m.group(2).strip()
                protos[m.group(1)] = 0 if args in ("", "void") else len(args.split(","))
    sigs = {n: at for n, _, at in xdg.SIGNATURES}
    assert set(protos) <= set(sigs)
    bad = {n: (k, len(sigs[n])) for n, k in protos.items() if len(sigs[n]) != k}
    assert not bad, bad
