"""The surrogate controller's trust policy (host logic only): which jumps are
judged by the plain LB, how the judging interval grows, and what a failed
judgement does.  The native jump is replaced by a scripted fake."""
import pytest

from paper_2405_14551_gb300 import surrogate as S


class _FakeSim:
    def __init__(self):
        self.h = object()
        self.steps = 0

    def step(self, n):
        self.steps += n


def _controller(monkeypatch, script):
    """A Controller with its lattices replaced by fakes; script: list of
    (accepted, judged error) the native cycle returns when judged."""
    calls = []

    def fake_cycle(h, judge, K, vol_tol, phi_tol):
        judged = judge is not None
        calls.append(judged)
        if not judged:
            return True, -1.0
        ok, err = script.pop(0)
        return ok, err

    monkeypatch.setattr(S.L, "lb_surrogate_cycle", fake_cycle)
    c = S.Controller.__new__(S.Controller)
    c.sim, c.K = _FakeSim(), 50
    c.shadow = _FakeSim()
    c.vol_tol, c.phi_tol = 0.02, 1e-2
    c.judge_every, c.backoff, c.judge_max, c.margin = 4, 8, 16, 0.75
    c.reset()
    return c, calls


def test_interval_grows_only_with_margin(monkeypatch):
    # passes: 0.009 (trust), 0.0082 (no margin), 0.007 (margin -> 8), 0.006 (-> 16), 0.005 (stays 16)
    c, calls = _controller(monkeypatch, [(True, 0.009), (True, 0.0082), (True, 0.007), (True, 0.006),
                                         (True, 0.005)])
    c.run(45)
    judged_at = [i for i, j in enumerate(calls) if j]
    assert judged_at == [0, 4, 8, 16, 32]
    assert c.interval == 16 and c.trusted and c.accepted == 45 and c.rejected == 0
    assert [e for _, e in c.judged] == [0.009, 0.0082, 0.007, 0.006, 0.005]


def test_failed_judgement_resets_and_suspends(monkeypatch):
    c, calls = _controller(monkeypatch, [(True, 0.005), (True, 0.005), (False, 0.02), (True, 0.009)])
    c.run(25)
    judged_at = [i for i, j in enumerate(calls) if j]
    # trust at jump 0, margin pass at jump 4 (-> 8), failure at jump 12 (cycle 12); 8 suspended
    # cycles without a jump, then every jump judged until one passes (jump 13, cycle 21)
    assert judged_at == [0, 4, 12, 13]
    assert c.rejected == 1 and c.interval == 4 and c.trusted
    assert len(calls) == 25 - 8
    # suspended cycles run 2K plain steps
    assert c.sim.steps == 25 * 50 + 8 * 50


def test_untrusted_controller_judges_every_jump(monkeypatch):
    c, calls = _controller(monkeypatch, [(False, 0.03)] * 3 + [(True, 0.004)] * 3)
    c.backoff = 0
    c.run(6)
    assert calls == [True] * 4 + [False] * 2  # trusted from the 4th jump on: every 4th judged
    assert c.interval == 4 and c.rejected == 3
