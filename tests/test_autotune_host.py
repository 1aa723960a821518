"""The autotuner's host logic on CPU: the schedule pick rule, the shape bucket and the
cached setting's application (no GPU: the network is a stand-in that records calls)."""
import json

from paper_2410_13055_gb300 import autotune


def _trial(b, w, ms):
    return {"bus_staged": b, "bat_warps": w, "ms_per_step": ms}


def test_pick_keeps_default_inside_the_margin():
    default = {"bus_staged": 1, "bat_warps": 2}
    trials = [_trial(0, 2, 10.0), _trial(1, 2, 10.1), _trial(2, 2, 9.95)]
    # 1.5 % faster than the default: inside a 2 % margin
    assert autotune.pick_schedule(trials, default, 0.02) == default
    # 5 % faster: taken
    trials[2]["ms_per_step"] = 9.6
    assert autotune.pick_schedule(trials, default, 0.02) == {"bus_staged": 2, "bat_warps": 2}
    # the default is the fastest
    assert autotune.pick_schedule([_trial(1, 2, 9.0), _trial(0, 1, 9.5)], default, 0.0) == default


def test_pick_without_a_timed_default_takes_the_fastest():
    default = {"bus_staged": 1, "bat_warps": 2}
    trials = [_trial(0, 1, 12.0), _trial(2, 1, 11.0)]
    assert autotune.pick_schedule(trials, default, 0.02) == {"bus_staged": 2, "bat_warps": 1}


class _FakeNet:
    def __init__(self, info, S):
        self.info, self.S = info, S
        self.calls = []

    def set_opts(self, **kw):
        self.calls.append(("set_opts", kw))

    def use_persistent(self, on):
        self.calls.append(("use_persistent", on))

    def set_schedule(self, **kw):
        self.calls.append(("set_schedule", kw))


def test_bucket_rounds_shapes_up_to_powers_of_two():
    assert autotune.bucket(_FakeNet([{"N": 100, "T": 168}] * 16, 16)) == "N128_T256_S16"
    # uneven batches take their largest network and horizon
    net = _FakeNet([{"N": 50, "T": 24}, {"N": 500, "T": 72}, {"N": 300, "T": 168}], 3)
    assert autotune.bucket(net) == "N512_T256_S4"
    assert autotune.bucket(_FakeNet([{"N": 1, "T": 1}], 1)) == "N1_T1_S1"


def test_load_applies_the_cached_setting(tmp_path):
    net = _FakeNet([{"N": 100, "T": 168}] * 16, 16)
    cache = tmp_path / "autotune.json"
    assert autotune.load(net, cache=str(cache)) is None and net.calls == []
    best = {"rho": 0.2, "check_every": 20, "persistent": False, "bus_staged": 1, "bat_warps": 2}
    cache.write_text(json.dumps({"N128_T256_S16": {"best": best, "time_s": 1.0, "trials": []},
                                 "N8_T32_S1": {"best": {"rho": 0.5}, "time_s": 1.0, "trials": []}}))
    assert autotune.load(net, cache=str(cache)) == best
    kinds = dict((k, v) for k, v in net.calls)
    assert kinds["set_opts"] == {"rho": 0.2, "check_every": 20}
    assert kinds["use_persistent"] is False
    assert kinds["set_schedule"] == {"bus_staged": 1, "bat_warps": 2}
    # another shape bucket: nothing applied
    other = _FakeNet([{"N": 5, "T": 24}], 2)
    assert autotune.load(other, cache=str(cache)) is None and other.calls == []


class _Event:
    """A stand-in for torch.cuda.Event that reads a fake clock."""
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self):
        self.t = _Event.clock[0]

    def elapsed_time(self, end):
        return end.t - self.t


class _StepNet:
    """A network stand-in whose step time depends on the schedule in force; the step
    advances the fake clock and perturbs the state, which the tuner must restore."""
    def __init__(self, times, default):
        import torch
        self.times, self.sched = times, dict(default)
        self.fwd, self.adj = torch.zeros(8), torch.ones(8)
        self.set_calls = []

    def schedule(self):
        return dict(self.sched)

    def set_schedule(self, **kw):
        self.sched = dict(kw)
        self.set_calls.append(dict(kw))

    def state(self, adjoint=False):
        return self.adj if adjoint else self.fwd

    def step(self, eta):
        _Event.clock[0] += self.times[(self.sched["bus_staged"], self.sched["bat_warps"])]
        self.fwd += 1.0
        self.adj -= 1.0
        eta += 0.5


def test_schedule_step_tuner_times_restores_and_picks(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    times = {(0, 2): 12.0, (0, 1): 13.0, (1, 2): 10.0, (1, 1): 11.0, (2, 2): 9.0, (2, 1): 10.5}
    net = _StepNet(times, {"bus_staged": 1, "bat_warps": 2})
    eta = torch.zeros(4)
    flushes = []
    out = autotune.tune_schedule_step(net, eta, step=net.step, steps=2, reps=2, margin=0.02,
                                      flush=lambda: flushes.append(1))
    got = {(t["bus_staged"], t["bat_warps"]): t["ms_per_step"] for t in out["trials"]}
    assert got == times
    assert out["default"] == {"bus_staged": 1, "bat_warps": 2}
    # 9.0 against the default's 10.0 is outside the 2 % margin
    assert out["best"] == {"bus_staged": 2, "bat_warps": 2} and net.schedule() == out["best"]
    # plan and iteration state are those of before the tuner
    assert torch.all(eta == 0) and torch.all(net.fwd == 0) and torch.all(net.adj == 1)
    assert len(flushes) == 6 * 2 * 2
    # a narrower gap stays with the default
    times[(2, 2)] = 9.9
    net = _StepNet(times, {"bus_staged": 1, "bat_warps": 2})
    out = autotune.tune_schedule_step(net, torch.zeros(4), step=net.step, steps=1, reps=1, margin=0.02)
    assert out["best"] == {"bus_staged": 1, "bat_warps": 2} and net.schedule() == out["best"]
