"""Failure detection on the GPU without faulting it.

Every failure here is made on the host or by a short device bound:
- an allocator hook (hp_set_allocator) that refuses the k-th workspace
  request: the call returns HP_ERR_OOM, every block it was given is handed
  back, and the next call (default allocator) is correct;
- the test-only option debug_walk_cap, which makes the matching's bounded
  tree walks give up early: the call returns HP_ERR_TIMEOUT before the level
  is contracted, and the context stays usable.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu

ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_20497_gb300 import build
    build.build()
    oracle.build()
    hp.load()
    return t


class Hook:
    """Counting allocator over torch's caching allocator; refuses the
    fail_at-th request (1-based) when set."""

    def __init__(self, torch, fail_at=None):
        self.torch, self.fail_at = torch, fail_at
        self.requests, self.frees, self.live = 0, 0, set()
        self._a, self._f = ALLOC_T(self.alloc), FREE_T(self.free)

    def alloc(self, size, ctx):
        self.requests += 1
        if self.fail_at is not None and self.requests == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(size, device=self.torch.cuda.current_device())
        self.live.add(p)
        return p

    def free(self, p, ctx):
        self.frees += 1
        self.live.remove(p)
        self.torch.cuda.caching_allocator_delete(p)

    def __enter__(self):
        rc = hp.load().hp_set_allocator(ctypes.cast(self._a, ctypes.c_void_p), ctypes.cast(self._f, ctypes.c_void_p),
                                        None)
        assert rc == hp.HP_OK
        return self

    def __exit__(self, *exc):
        assert hp.load().hp_set_allocator(None, None, None) == hp.HP_OK
        return False


def _graph():
    return inputs.random_snn(2048, 31, seed=5), 128, 512


def _matches_oracle(g, omega, delta, r):
    o = oracle.partition(g, omega, delta, seed=1)
    assert r.status == hp.HP_OK, hp.hp_last_error()
    assert np.array_equal(r.part, o.part)


def test_allocator_hook_sees_every_block_back(torch):
    g, omega, delta = _graph()
    with Hook(torch) as h:
        r = hp.partition(g, omega, delta, seed=1)
    assert h.requests > 10 and h.live == set() and h.frees == h.requests
    _matches_oracle(g, omega, delta, r)


@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5, 0.9, 1.0])
def test_refused_allocation_returns_oom_and_frees_everything(torch, frac):
    g, omega, delta = _graph()
    with Hook(torch) as probe:
        hp.partition(g, omega, delta, seed=1)
    k = 1 + int(frac * (probe.requests - 1))
    with Hook(torch, fail_at=k) as h:
        r = hp.partition(g, omega, delta, seed=1)
    assert r.status == hp.HP_ERR_OOM, (k, r.status, hp.hp_last_error())
    assert "allocation" in hp.hp_last_error()
    assert h.requests == k and h.live == set() and h.frees == k - 1
    # the next call, with the default allocator, is unaffected
    _matches_oracle(g, omega, delta, hp.partition(g, omega, delta, seed=1))


def test_bounded_walk_gives_up_with_timeout(torch):
    g, omega, delta = _graph()
    # precondition: the first proposal graph has a path of at least three
    # proposal edges that ends at a root, so a walk of one step cannot finish
    cand, _ = oracle.propose(g, np.ones(g.num_nodes, np.int32), omega, delta, seed=1, level=0, pi=4)
    t = cand[:, 0]

    def depth(v):
        d = 0
        while t[v] >= 0 and t[t[v]] != v and d <= g.num_nodes:
            v, d = t[v], d + 1
        return d
    assert max(depth(v) for v in range(g.num_nodes)) >= 3
    r = hp.partition(g, omega, delta, seed=1, debug_walk_cap=1)
    assert r.status == hp.HP_ERR_TIMEOUT, (r.status, hp.hp_last_error())
    assert "coarsening level 0" in hp.hp_last_error()
    # the context is intact: a normal call afterwards is bit-exact
    _matches_oracle(g, omega, delta, hp.partition(g, omega, delta, seed=1))
    # a cap at least as deep as every walk changes nothing
    _matches_oracle(g, omega, delta, hp.partition(g, omega, delta, seed=1, debug_walk_cap=g.num_nodes))


def test_walk_cap_option_is_checked(torch):
    g, omega, delta = _graph()
    r = hp.partition(g, omega, delta, seed=1, debug_walk_cap=-1)
    assert r.status == hp.HP_ERR_INVALID_ARG
