"""Host logic of bench.py that needs no GPU: the default workload is the full emission batch, ranks get
distinct packet streams of the same jobs, every workload has an oracle sample, and the clock record
is summarised as the timing rules read it."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _args(bench, monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


def test_default_run_is_the_full_emission_batch(bench, monkeypatch):
    a = _args(bench, monkeypatch)
    assert a.gpus == 1 and a.warmup >= 3 and a.impl == "gcmc" and a.workload == "emission"
    w0, w1 = bench.workload(a, 0), bench.workload(a, 1)
    g = w0.grid
    assert (g.nlon, g.nlat, g.nr) == (128, 64, 50)
    assert len(w0.jobs) == 240 and all(j.n_packets == 1_000_000 for j in w0.jobs)
    # weak scaling: each rank runs the same jobs on its own packet streams
    assert [j.key for j in w0.jobs] == [j.key for j in w1.jobs] and w0.seed != w1.seed


@pytest.mark.parametrize("name,n_jobs", [("albedo", 1), ("phasecurve", 960), ("band", 30), ("emission-hires", 954)])
def test_other_workloads(bench, monkeypatch, name, n_jobs):
    a = _args(bench, monkeypatch, "--workload", name)
    assert len(bench.workload(a, 0).jobs) == n_jobs


def test_forced_and_continuous_absorption_flags(bench, monkeypatch):
    a = _args(bench, monkeypatch, "--workload", "phasecurve", "--forced-first", "--cont-abs")
    wl = bench.workload(a, 0)
    assert wl.source.opts.forced_first == 1 and wl.source.opts.cont_abs == 1
    assert wl.name.endswith("_forced_contabs")


def test_every_workload_has_an_oracle_sample(bench, monkeypatch):
    a = _args(bench, monkeypatch)
    choices = {"emission", "albedo", "phasecurve", "transmission", "transit-scatter", "band", "emission-hires"}
    assert set(bench.CPU_SAMPLE) == choices and set(bench.REF_SAMPLE) == choices
    assert a.workload in bench.CPU_SAMPLE


def test_clock_summary(bench):
    c = bench.ClockSampler(None)
    c.out = ("2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active\n"
             "2055, 2070, 1380.0, Not Active, Not Active, Not Active, Active\n"
             "2040, 2070, 1395.2, Not Active, Not Active, Not Active, Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.out = "2070, 2070, 900.1, Active, Not Active, Active, Not Active\n"
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.out = ""
    assert c.summary()["reasons"] == ["unsampled"]
