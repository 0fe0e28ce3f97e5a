"""Host-side pieces of bench.py that need no GPU: the oracle's GMG sample of
the CPU baseline converges on a small level and reports what it ran, and the
clock sampler's parser reads nvidia-smi's CSV (median SM clock, the throttle
reasons that were active), and the sampler names the GPU by its UUID when
nvidia-smi accepts it, else by torch's index; the bench command lines quoted
in the committed profile summaries parse with the current bench.py."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_gmg_sample_converges_and_labels_the_extrapolation():
    g = bench.cpu_baseline_gmg(level=2)
    assert g["kind"] == "oracle" and g["level"] == 2
    assert g["unique_dofs"] == (4 * 4 + 1) ** 3
    assert g["rel_res"] <= 1e-8 and 5 <= g["v_cycles"] <= 60
    assert g["level6_solve_s_extrapolated"] == pytest.approx(
        g["solve_s"] * (4 * 64 + 1) ** 3 / g["unique_dofs"])
    assert "extrapolated" in g["sample"]


def test_clock_sampler_parses_nvidia_smi_csv(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clk.csv")
    with open(c.path, "w") as f:
        f.write("0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1995, 2070, 990.2, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("garbage line\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.f = open(os.devnull, "w")
    r = c.stop()
    assert r == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_names_the_gpu_by_uuid_when_nvidia_smi_accepts_it(monkeypatch):
    torch = pytest.importorskip("torch")

    class Props:
        uuid = "3f1c2a9e-0000-1111-2222-333344445555"

    class Result:
        def __init__(self, rc, out):
            self.returncode, self.stdout = rc, out

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: Props())
    calls = []

    def accepts(cmd, **kw):
        calls.append(cmd)
        return Result(0, "5\n")

    gid = bench.ClockSampler.smi_gpu_id(0, run=accepts)
    assert gid == "GPU-3f1c2a9e-0000-1111-2222-333344445555"
    assert calls[0][1] == f"--id={gid}"
    # nvidia-smi refuses the id (or is missing): the torch index is kept
    assert bench.ClockSampler.smi_gpu_id(2, run=lambda cmd, **kw: Result(6, "")) == "2"

    def missing(cmd, **kw):
        raise FileNotFoundError("nvidia-smi")

    assert bench.ClockSampler.smi_gpu_id(1, run=missing) == "1"


def test_clock_sampler_falls_back_to_the_index_without_device_properties(monkeypatch):
    torch = pytest.importorskip("torch")

    def no_gpu(i):
        raise RuntimeError("no CUDA device")

    monkeypatch.setattr(torch.cuda, "get_device_properties", no_gpu)
    assert bench.ClockSampler.smi_gpu_id(3) == "3"


def _profile_commands():
    """Every `python bench.py ...` command quoted in profiles/*.md, with
    backslash continuations joined and redirections dropped."""
    import glob
    import shlex
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            at = line.find("python bench.py")
            if at < 0:
                continue
            words = shlex.split(line[at:].split(">")[0].split("&&")[0])
            out.append((os.path.basename(path), words[2:]))
    return out


def test_profile_command_lines_parse_with_the_current_bench():
    cmds = _profile_commands()
    assert len(cmds) >= 6
    ap = bench.make_parser()
    for name, argv in cmds:
        args = ap.parse_args(argv)
        assert args.impl == "gb300", name


def test_only_keeps_the_named_legs_and_every_leg_has_a_switch():
    import bench
    ap = bench.make_parser()
    for leg in bench.LEGS:
        assert hasattr(ap.parse_args([]), "no_" + leg), leg
        assert getattr(ap.parse_args([]), "no_" + leg) is False
    a = bench.apply_only(ap.parse_args(["--only", "gmg,kernels"]))
    assert not a.no_gmg and not a.no_kernels
    assert all(getattr(a, "no_" + leg) for leg in bench.LEGS if leg not in ("gmg", "kernels"))
    a = bench.apply_only(ap.parse_args(["--only", "headline"]))
    assert all(getattr(a, "no_" + leg) for leg in bench.LEGS)
    a = bench.apply_only(ap.parse_args([]))
    assert not any(getattr(a, "no_" + leg) for leg in bench.LEGS)
