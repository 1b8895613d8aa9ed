"""CPU checks of the C ABI: the library builds, loads, and exports every symbol include/kpp.h declares.

No compute call is made here (there is no GPU); only host-only entry points are called.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_11673_gb300 import build as kbuild
from paper_2501_11673_gb300 import kpp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "kpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("kpp_", "cdpp_"))))


@pytest.fixture(scope="module")
def lib():
    path = kbuild.build()
    return kpp.load(path)


def test_header_declarations_are_all_exported(lib):
    declared = _declared_functions()
    assert "kpp_solve" in declared and "cdpp_solve" in declared and "kpp_factor_blocks" in declared
    assert "kpp_partition" in declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in kpp.h but not exported"
    assert sorted(kpp.EXPORTS) == declared


def test_host_only_entry_points(lib):
    p = lib.kpp_params_default()
    assert p.tol == 1e-8 and p.adaptive_rho == 1 and p.max_outer == 20
    assert lib.kpp_status_string(0) == b"KPP_OK"
    assert lib.kpp_status_string(4) == b"KPP_ERR_NOT_SPD"
    P = kpp.Partition(103, 10)
    assert P.nb == 11
    h = ctypes.c_void_p()
    assert lib.kpp_partition(0, 10, ctypes.byref(h)) == kpp.ERR_ARG
    assert lib.kpp_partition(10, 0, ctypes.byref(h)) == kpp.ERR_ARG
    assert "kpp_partition" in kpp.last_error()
    assert kpp.build_info().startswith("sm_103a")


def test_build_targets_sm_103a_only():
    assert kbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_plan_handles_and_tune_cache_on_the_host(lib, tmp_path):
    """Null plan handles are refused without touching the device; the autotuner cache file round-trips
    and a malformed file loads nothing."""
    assert lib.kpp_plan_launch(None, None) == kpp.ERR_ARG
    assert lib.kpp_plan_report(None, None, None) == kpp.ERR_ARG
    assert lib.kpp_plan_info(None, None, None, None) == kpp.ERR_ARG
    lib.kpp_plan_destroy(None)
    kpp.tune_cache_clear()
    assert kpp.tune_cache_size() == 0
    good = tmp_path / "cache.txt"
    good.write_text("# comment\nsm103-n152:r4096:c4096:d0:s64:k1:m1:n1:v3 3 96\nsm103-n152:r10:c10:d1:s2:k1:m0:n1:v3 2 1\n")
    kpp.tune_cache_load(good)
    assert kpp.tune_cache_size() == 2
    out = tmp_path / "out.txt"
    kpp.tune_cache_save(out)
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert sorted(lines) == sorted(["sm103-n152:r4096:c4096:d0:s64:k1:m1:n1:v3 3 96",
                                    "sm103-n152:r10:c10:d1:s2:k1:m0:n1:v3 2 1"])
    kpp.tune_cache_clear()
    bad = tmp_path / "bad.txt"
    bad.write_text("key 3 96\nkey2 7 1\n")  # generation 7 does not exist
    with pytest.raises(kpp.KppError):
        kpp.tune_cache_load(bad)
    assert kpp.tune_cache_size() == 0
    with pytest.raises(kpp.KppError):
        kpp.tune_cache_load(tmp_path / "missing.txt")


def test_hadamard_entry_points_refuse_bad_arguments_on_the_host(lib):
    """kpp_rht_forward / kpp_rht_inverse check sizes, dtype and pointers before any device work."""
    m = kpp.Matrix(ctypes.c_void_p(16), kpp.KPP_F64, 0, 8, 8, 8)
    vp = ctypes.c_void_p
    for n in (0, 6, 12, 1 << 15):  # not a power of 2, or above 16384
        assert lib.kpp_rht_forward(n, vp(16), ctypes.byref(m), vp(16), None, None, 0, None) == kpp.ERR_ARG
        assert "power of 2" in kpp.last_error()
    m6 = kpp.Matrix(ctypes.c_void_p(16), kpp.KPP_F64, 0, 4, 8, 8)  # rows != n
    assert lib.kpp_rht_forward(8, vp(16), ctypes.byref(m6), vp(16), None, None, 0, None) == kpp.ERR_ARG
    m32 = kpp.Matrix(ctypes.c_void_p(16), kpp.KPP_F32, 0, 8, 8, 8)  # not FP64
    assert lib.kpp_rht_forward(8, vp(16), ctypes.byref(m32), vp(16), None, None, 0, None) == kpp.ERR_ARG
    assert lib.kpp_rht_forward(8, None, ctypes.byref(m), vp(16), None, None, 0, None) == kpp.ERR_ARG
    assert lib.kpp_rht_forward(8, vp(16), ctypes.byref(m), vp(16), None, None, 2, None) == kpp.ERR_ARG  # k > 0, no b
    assert lib.kpp_rht_inverse(8, vp(16), vp(16), vp(16), 0, None) == kpp.ERR_ARG                   # k < 1
    assert lib.kpp_rht_inverse(6, vp(16), vp(16), vp(16), 1, None) == kpp.ERR_ARG
    assert lib.kpp_rht_inverse(8, vp(16), None, vp(16), 1, None) == kpp.ERR_ARG


def _oracle_memo_sequence(seed, sys_id, cd, rows, cols, s, t0, count, nb0):
    import oracle
    nb, blocks, subsets = nb0, [], []
    for t in range(t0, t0 + count):
        j = oracle.memo_draw(seed, t, sys_id, cd, rows, cols, s, nb)
        if j < 0:
            subsets.append(oracle.memo_subset(seed, t, sys_id, rows, s))
            j, nb = nb, nb + 1
        blocks.append(j)
    return blocks, subsets, nb


@pytest.mark.parametrize("cd,rows,cols,s,seed,sys_id", [(True, 256, 256, 16, 11, 0), (True, 4096, 4096, 64, 1, 3),
                                                        (False, 2000, 200, 20, 0, 5), (False, 500, 900, 7, 2**63 + 9, 1)])
def test_memo_sequence_matches_the_oracle_draws(lib, cd, rows, cols, s, seed, sys_id):
    """The library's host draw of the memo block sequence (kpp_memo_sequence) equals the oracle's, step by
    step and subset by subset (integer results: bitwise), and a window split in two gives the same
    sequence as one window."""
    T = 3000
    blocks, subsets, nb = kpp.memo_sequence(seed, sys_id, cd, rows, cols, s, 0, T)
    ob, osub, onb = _oracle_memo_sequence(seed, sys_id, cd, rows, cols, s, 0, T, 0)
    assert nb == onb and blocks.tolist() == ob
    assert len(subsets) == len(osub) and all((a == b).all() for a, b in zip(subsets, osub))
    b1, s1, nb1 = kpp.memo_sequence(seed, sys_id, cd, rows, cols, s, 0, 1234)
    b2, s2, nb2 = kpp.memo_sequence(seed, sys_id, cd, rows, cols, s, 1234, T - 1234, nb1)
    assert nb2 == nb and (np.concatenate([b1, b2]) == blocks).all()
    assert (np.concatenate([s1, s2]) == subsets).all()


def test_memo_sequence_refuses_bad_arguments(lib):
    nb = ctypes.c_int64()
    p = ctypes.POINTER(ctypes.c_int64)
    buf = np.zeros(64, dtype=np.int64)
    args = lambda mode, rows, cols, s, count, cap: (1, 0, mode, rows, cols, s, 0, count, 0, buf.ctypes.data_as(p),
                                                    buf.ctypes.data_as(p), cap, ctypes.byref(nb))
    assert lib.kpp_memo_sequence(*args(2, 10, 10, 2, 4, 4)) == kpp.ERR_ARG   # mode
    assert lib.kpp_memo_sequence(*args(1, 10, 12, 2, 4, 4)) == kpp.ERR_ARG   # CD++ needs a square matrix
    assert lib.kpp_memo_sequence(*args(0, 10, 12, 11, 4, 4)) == kpp.ERR_ARG  # s > rows
    assert lib.kpp_memo_sequence(*args(0, 10, 12, 2, 4, 1)) == kpp.ERR_ARG   # steps 0, 1 both draw new blocks
    assert nb.value == 1 and "subsets_cap" in kpp.last_error()


def test_solver_entry_points_refuse_bad_arguments_on_the_host(lib):
    """The factor, solve, batched, plan, server, sampling, Gram and residual entry points check their
    arguments before any device work: each call below has exactly one bad argument (the device pointers
    are never dereferenced) and returns KPP_ERR_ARG with a message."""
    vp = ctypes.c_void_p
    dev = vp(256)  # a stand-in device address; validation rejects every call before using it
    P = kpp.Partition(64, 8)
    out = vp()
    prm = kpp.params(lam=1e-3)
    rep = kpp.Report()

    def mat(rows=64, cols=64, dtype=kpp.KPP_F64, ld=None, data=dev):
        return kpp.Matrix(data, dtype, 0, rows, cols, cols if ld is None else ld)

    fb = lib.kpp_factor_blocks
    assert fb(ctypes.byref(mat()), P.handle, 1e-3, 0, None, None) == kpp.ERR_ARG              # no output handle
    assert fb(ctypes.byref(mat()), None, 1e-3, 0, ctypes.byref(out), None) == kpp.ERR_ARG  # no partition
    assert fb(ctypes.byref(mat(dtype=7)), P.handle, 1e-3, 0, ctypes.byref(out), None) == kpp.ERR_ARG
    assert fb(ctypes.byref(mat(ld=32)), P.handle, 1e-3, 0, ctypes.byref(out), None) == kpp.ERR_ARG  # ld < cols
    assert fb(ctypes.byref(mat(data=None)), P.handle, 1e-3, 0, ctypes.byref(out), None) == kpp.ERR_ARG
    assert fb(ctypes.byref(mat(rows=63)), P.handle, 1e-3, 0, ctypes.byref(out), None) == kpp.ERR_ARG  # rows != partition
    assert fb(ctypes.byref(mat()), P.handle, 1e-3, 2, ctypes.byref(out), None) == kpp.ERR_ARG         # mode
    assert fb(ctypes.byref(mat()), P.handle, -1.0, 0, ctypes.byref(out), None) == kpp.ERR_ARG          # lambda < 0
    assert fb(ctypes.byref(mat()), P.handle, float("nan"), 0, ctypes.byref(out), None) == kpp.ERR_ARG
    assert fb(ctypes.byref(mat(cols=32)), P.handle, 1e-3, 1, ctypes.byref(out), None) == kpp.ERR_ARG  # CD++ not square
    assert "kpp_factor_blocks" in kpp.last_error()

    for f in (lib.kpp_solve, lib.cdpp_solve, lib.cdpp_solve_noalloc):  # no factors
        assert f(ctypes.byref(mat()), dev, dev, P.handle, None, ctypes.byref(prm), ctypes.byref(rep), None) == kpp.ERR_ARG
    assert lib.kpp_solve(ctypes.byref(mat()), None, dev, P.handle, dev, ctypes.byref(prm), ctypes.byref(rep),
                         None) == kpp.ERR_ARG                                                  # no b
    Bs, Xs, Fs = (vp * 1)(dev), (vp * 1)(dev), (vp * 1)(None)
    for f in (lib.kpp_solve_batched, lib.cdpp_solve_batched):
        assert f(0, ctypes.byref(mat()), Bs, Xs, 1, P.handle, Fs, ctypes.byref(prm), ctypes.byref(rep), None) == kpp.ERR_ARG
        assert f(1, ctypes.byref(mat()), Bs, Xs, 33, P.handle, Fs, ctypes.byref(prm), ctypes.byref(rep), None) == kpp.ERR_ARG
    assert lib.kpp_plan_create(1, ctypes.byref(mat()), Bs, Xs, 1, P.handle, Fs, ctypes.byref(prm), 2, None,
                               ctypes.byref(out)) == kpp.ERR_ARG                               # mode
    assert lib.kpp_plan_create(1, ctypes.byref(mat()), Bs, Xs, 1, P.handle, Fs, ctypes.byref(prm), 0, None,
                               ctypes.byref(out)) == kpp.ERR_ARG                               # no factors
    assert lib.kpp_server_create(0, 4, 0, ctypes.byref(out)) == kpp.ERR_ARG                    # no budget
    assert lib.kpp_server_create(1 << 30, 0, 0, ctypes.byref(out)) == kpp.ERR_ARG              # no slots
    assert lib.kpp_server_create(1 << 30, 65, 0, ctypes.byref(out)) == kpp.ERR_ARG
    assert lib.kpp_server_create(1 << 30, 4, 65, ctypes.byref(out)) == kpp.ERR_ARG             # slot width
    assert lib.kpp_sample_blocks(1, 0, 0, 10, 0, dev, None) == kpp.ERR_ARG                     # nb < 1
    assert lib.kpp_sample_blocks(1, 0, 0, -1, 4, dev, None) == kpp.ERR_ARG
    assert lib.kpp_sample_blocks(1, 0, 0, 10, 4, None, None) == kpp.ERR_ARG
    for v in (0, 4):
        assert lib.kpp_set_kernel_variant(v) == kpp.ERR_ARG
    used = ctypes.c_int32()
    assert lib.kpp_block_gram(ctypes.byref(mat()), 0, 0.0, 0, dev, ctypes.byref(used), None) == kpp.ERR_ARG
    assert lib.kpp_block_gram(ctypes.byref(mat()), 2000, 0.0, 0, dev, ctypes.byref(used), None) == kpp.ERR_ARG
    assert lib.kpp_block_gram(ctypes.byref(mat()), 8, 0.0, 4, dev, ctypes.byref(used), None) == kpp.ERR_ARG
    assert lib.kpp_block_gram(ctypes.byref(mat()), 8, 0.0, 0, None, ctypes.byref(used), None) == kpp.ERR_ARG
    r = ctypes.c_double()
    assert lib.kpp_rel_residual(ctypes.byref(mat()), dev, dev, None, None) == kpp.ERR_ARG
    assert lib.kpp_rel_residual(ctypes.byref(mat()), None, dev, ctypes.byref(r), None) == kpp.ERR_ARG
    hb = np.zeros(64)
    assert lib.kpp_solve_host(ctypes.byref(mat()), hb.ctypes.data, hb.ctypes.data, 8, 2, ctypes.byref(prm),
                              ctypes.byref(rep), None) == kpp.ERR_ARG                          # mode
    assert kpp.last_error() != ""


def test_binding_structs_match_the_c_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C compiler gives the
    header's struct (gcc on include/kpp.h), so no field is read or written at the wrong place."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"kpp_matrix": (kpp.Matrix, ["data", "dtype", "reserved", "rows", "cols", "ld"]),
               "kpp_params": (kpp.Params, ["lambda", "tol", "max_iters", "seed", "sys_id", "adaptive_rho", "rho0",
                                           "eta", "grid", "refine", "max_outer", "reserved0", "inner_tol",
                                           "reserved1"]),
               "kpp_report": (kpp.Report, ["iters", "outer", "rel_res_true", "rel_res_est", "rho_final", "status",
                                           "bad_block", "device_ms", "kernel_ms", "launches", "reserved"]),
               "kpp_serving_stats": (kpp.ServingStats, ["completed", "failed", "p50_ms", "p99_ms", "max_ms",
                                                        "solves_per_s", "span_s", "peak_bytes", "budget_bytes",
                                                        "loop_launches", "loop_slots", "reserved"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kpp.h"', "int main(void) {"]
    for cname, (_, fields) in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, (cls, fields) in structs.items():
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        pyfields = [f for f, _ in cls._fields_]
        assert len(pyfields) == len(fields), cname
        for pf, cf in zip(pyfields, fields):
            assert getattr(cls, pf).offset == got[(cname, cf)], (cname, cf)
