"""A context is destroyed only after every handle made with it, whatever order
the garbage collector finalizes them in (runs without a GPU: the library
calls are replaced by recorders)."""
import gc

import pytest

from paper_2510_23679_gb300 import pd


class _FakeLib:
    def __init__(self):
        self.log = []
        self.destroyed = set()

    def pd_ctx_destroy(self, h):
        self.log.append(("ctx", h))
        self.destroyed.add(h)

    def pd_profiles_free(self, h):
        assert "ctx" not in self.destroyed, "handle freed after its context"
        self.log.append(("profiles", h))


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(pd, "_lib", lib)
    return lib


def _ctx():
    c = pd.Ctx.__new__(pd.Ctx)
    c.handle = "ctx"
    return c


def test_close_waits_for_live_handles(fake):
    c = _ctx()
    a, b = pd.Profiles(c, "p1"), pd.Profiles(c, "p2")
    c.close()
    assert fake.log == []
    a.free()
    assert fake.log == [("profiles", "p1")]
    b.free()
    assert fake.log == [("profiles", "p1"), ("profiles", "p2"), ("ctx", "ctx")]
    c.close()
    assert len(fake.log) == 3


def test_cycle_finalized_in_any_order(fake):
    gc.collect()
    gc.disable()
    try:
        c = _ctx()
        box = {"ctx": c, "handles": [pd.Profiles(c, f"p{i}") for i in range(4)]}
        box["self"] = box  # a cycle holding the context and its handles
        c.cycle = box
        del c, box
        gc.collect()
    finally:
        gc.enable()
    assert sorted(fake.log[:-1]) == [("profiles", f"p{i}") for i in range(4)]
    assert fake.log[-1] == ("ctx", "ctx")
