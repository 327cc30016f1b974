"""The C-ABI library builds, loads and exports every symbol include/hp.h
declares; host-only calls work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2605_20497_gb300 import build, hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hp.load()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "hp_partition" in syms and "hp_partition_host" in syms
    for s in syms:
        assert hasattr(lib, s), s
        assert s in hp.EXPORTS, s


def test_only_declared_symbols_are_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", hp.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    ours = {s for s in exported if s.startswith("hp_")}
    assert ours == set(declared_symbols())


def test_host_only_calls(lib):
    o = hp.hp_default_options()
    assert (o.pi, o.theta, o.chain_window, o.chain_rounds, o.noise_permille, o.count_kind, o.max_levels,
            o.debug_table_cap, o.learned_k) == (4, 16, 256, 16, 100, 0, 256, 0, 0)
    assert not o.merge_model
    assert hp.hp_status_string(hp.HP_OK) == "ok"
    assert "CSR" in hp.hp_status_string(hp.HP_ERR_BAD_CSR)
    assert hp.hp_last_error() == ""


def test_argument_checks_before_any_device_work(lib):
    # these return before touching CUDA, so they run without a GPU
    assert lib.hp_partition_batch(None, 0, None, 4, None, None, None) == hp.HP_OK
    assert lib.hp_partition_batch(None, 1, None, 4, None, None, None) == hp.HP_ERR_INVALID_ARG
    one = (hp.hp_instance * 1)()
    assert lib.hp_partition_batch(one, 1, None, -1, None, None, None) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_partition_batch(one, 1, None, 65, None, None, None) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_connectivity_noalloc(None, None, -1, None, None, 0, 0, None, None, None) == hp.HP_ERR_INVALID_ARG
    assert hp.hp_last_error() == "invalid argument"
    assert lib.hp_batch_tuned_concurrency(0, 99) == 0 and lib.hp_batch_tuned_concurrency(-1, 0) == 0


def test_struct_layout_matches_header(lib):
    assert ctypes.sizeof(hp.hp_options) == 10 * 4 + 8 + 8
    assert ctypes.sizeof(hp.hp_merge_model) == 64 * 16 + 64 * 64 + 64 + 4 * (64 + 64 + 3)
    assert ctypes.sizeof(hp.hp_stats) == 8 + 8 + 6 * 4 + 8 + 8 + 3 * 8 + 3 * 8 + 8 + 8
    assert ctypes.sizeof(hp.hp_level_trace) == 4 * 4 + 3 * 8 + 6 * 4
    assert ctypes.sizeof(hp.hp_instance) == 4 * 8 + 4 * 4 + 8 + 8


def test_learned_priority_checks_before_any_device_work(lib):
    from paper_2605_20497_gb300 import inputs
    good = hp.merge_model(inputs.random_merge_model(0))
    bad = hp.merge_model(inputs.random_merge_model(0))
    bad.w2[17] = -128
    assert lib.hp_merge_scores(None, 0, ctypes.byref(good), None, None) == hp.HP_OK
    assert lib.hp_merge_scores(None, -1, ctypes.byref(good), None, None) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_merge_scores(None, 0, ctypes.byref(bad), None, None) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_merge_scores(None, 5, ctypes.byref(good), None, None) == hp.HP_ERR_INVALID_ARG
    off = (ctypes.c_int32 * 1)(0)   # a valid empty hypergraph: only the options are wrong
    for kw in (dict(learned_k=16), dict(learned_k=3, model=inputs.random_merge_model(0)),
               dict(learned_k=17, model=inputs.random_merge_model(0))):
        o = hp.options(**kw)
        st = hp.hp_stats()
        assert lib.hp_partition(None, off, 0, 0, None, None, 4, 4, 0, ctypes.byref(o), None,
                                ctypes.byref(st), None) == hp.HP_ERR_INVALID_ARG, kw
    m = inputs.random_merge_model(0)
    m.shift2 = 31
    o = hp.options(learned_k=16, model=m)
    st = hp.hp_stats()
    assert lib.hp_partition(None, off, 0, 0, None, None, 4, 4, 0, ctypes.byref(o), None, ctypes.byref(st),
                            None) == hp.HP_ERR_INVALID_ARG
