"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports is tied to the sources it was
captured on (profiles/*.md list the kernel's source files and the sha256 of their bytes), and the figures the
line derives from event times."""
import hashlib
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = {
    ("k_emit_recon_u8", None),
    ("k_batch_tiles", "batch256_portraits_512to4096_matte_b6_b20"),
    ("k_soft_bwd", "soft32_3x1024x1024_f32_b8_b16"),
}


def _fields(path):
    vals = {}
    for line in open(path).read().splitlines():
        if line.strip().startswith("- ") and ":" in line:
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


@pytest.mark.parametrize("kernel,workload", sorted(PROFILES, key=str))
def test_profile_summaries_name_their_sources(kernel, workload):
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload or bench.WORKLOAD))
    vals = _fields(path)
    srcs = [s.strip() for s in vals["source_files"].split(",")]
    assert srcs and all(os.path.exists(os.path.join(ROOT, s)) for s in srcs)
    assert len(vals["sources_sha256"]) == 64
    assert int(vals["dram_bytes_per_launch_full_workload"]) > 0


def test_traffic_follows_the_sources(tmp_path, monkeypatch):
    """A copy of the tree whose profile hash matches its sources reports the traffic; one changed source byte
    turns it into null."""
    kernel, workload = "k_emit_recon_u8", bench.WORKLOAD
    name = "%s_%s.md" % (kernel, workload)
    vals = _fields(os.path.join(ROOT, "profiles", name))
    srcs = [s.strip() for s in vals["source_files"].split(",")]
    (tmp_path / "profiles").mkdir()
    for s in srcs:
        dst = tmp_path / s
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(ROOT, s), dst)
    h = hashlib.sha256()
    for s in srcs:
        h.update((tmp_path / s).read_bytes())
    text = open(os.path.join(ROOT, "profiles", name)).read()
    text = text.replace(vals["sources_sha256"], h.hexdigest())
    (tmp_path / "profiles" / name).write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile(kernel) == int(vals["dram_bytes_per_launch_full_workload"])
    last = tmp_path / srcs[-1]
    last.write_bytes(last.read_bytes() + b"\n")
    assert bench.traffic_from_profile(kernel) is None
    assert bench.traffic_from_profile("k_not_profiled") is None


def test_whole_job_throughput_counts_every_rank():
    one = bench.whole_job_mpx_per_s(1, 0.2)
    assert one == pytest.approx(bench.F * bench.M * bench.N / 1e6 / 0.2e-3)
    assert bench.whole_job_mpx_per_s(4, 0.2) == pytest.approx(4 * one)
