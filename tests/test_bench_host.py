"""Host logic of bench.py: the filter's roofline bound per width, the code
digest that ties a committed ncu summary to the filter source, and the
reading of the per-launch DRAM traffic from such a summary."""
import os
import shutil

import pytest

import bench


def test_filter_bound_per_width():
    # 148 SMs x 2032 MHz x min(16 / POPC, 64 / LOP3) for the (POPC, LOP3) mix per pair
    assert bench.filter_bound(64, 148, 2032.0) == pytest.approx(148 * 8 * 2032e6)
    assert bench.filter_bound(128, 148, 2032.0) == pytest.approx(148 * 16 / 3 * 2032e6)
    assert bench.filter_bound(256, 148, 2032.0) == pytest.approx(148 * 4 * 2032e6)
    # the binding pipe: XU at b = 64 and 128, both pipes equal at b = 256
    for b in (64, 128):
        popc, lop = bench.FILTER_MIX[b]
        assert 16 / popc < 64 / lop
    popc, lop = bench.FILTER_MIX[256]
    assert 16 / popc == 64 / lop


def test_folded_filter_bound():
    # b = 128 with the folded test: (2 + 3f) POPC and (2.4 + 6f) LOP3 per pair for a
    # fraction f of full-test steps; XU-bound for every f in [0, 1]; b = 256: (3 + 4f,
    # 7 + 16f)
    assert bench.filter_mix(128, 0.0) == (2, 2.4)
    assert bench.filter_mix(128, 1.0) == (5, 8.4)
    assert bench.filter_mix(256, 0.5) == (5, 15)
    assert bench.filter_mix(128) == bench.FILTER_MIX[128]
    assert bench.filter_mix(64, 0.5) == bench.FILTER_MIX[64]
    assert bench.filter_bound(128, 148, 2032.0, 0.0) == pytest.approx(148 * 8 * 2032e6)
    assert bench.filter_bound(128, 148, 2032.0, 1.0) == pytest.approx(148 * 16 / 5 * 2032e6)
    f = 0.046
    assert bench.filter_bound(128, 148, 2032.0, f) == pytest.approx(148 * 16 / (2 + 3 * f) * 2032e6)
    r = bench.filter_roofline(128, 1.0e12, 500.0, 148, 2032.0, full_frac=f)
    assert r["achieved"] == pytest.approx(2.0, abs=1e-4)
    assert r["frac"] == pytest.approx(2.0e12 / bench.filter_bound(128, 148, 2032.0, f), abs=1e-4)
    assert r["frac_of_full_test_bound"] == pytest.approx(2.0e12 / bench.filter_bound(128, 148, 2032.0),
                                                         abs=1e-4)


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // one\n'
           'const char *s = "x // not a comment /* nor this */";\n'
           '/* block\n comment */ char c = \'/\'; char d = \'\\\'\';\n'
           'int   b  =\n\n 2;')
    out = bench.strip_comments(src)
    assert "one" not in out and "block" not in out
    assert '"x // not a comment /* nor this */"' in out
    assert "char c = '/';" in out and "char d = '\\'';" in out
    assert out.endswith("int b = 2;")
    # layout and comments do not change the result, code does
    assert bench.strip_comments("int a=1;  /* x */\n// y\n") == bench.strip_comments("int a=1;")
    assert bench.strip_comments("int a=1;") != bench.strip_comments("int a=2;")


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_1711_07295_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("filter_core.cuh", "kernels.cuh", "filter.cu"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1711_07295_b300", "csrc", name), csrc / name)
    (root / "profiles").mkdir()
    return root, csrc


def test_digest_follows_code_not_comments(tmp_path, monkeypatch):
    root, csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.filter_source_digest()
    with open(csrc / "kernels.cuh", "a") as f:
        f.write("\n// a comment added at the end\n/* and a block */\n")
    assert bench.filter_source_digest() == d0
    with open(csrc / "kernels.cuh", "a") as f:
        f.write("constexpr int kAnotherConstant = 3;\n")
    assert bench.filter_source_digest() != d0


def test_profile_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    root, csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    digest = bench.filter_source_digest()
    prof = root / "profiles" / "filter_test.md"
    prof.write_text(f"# x\n\nfilter source sha256[:16]: {digest}\n\n"
                    "dram bytes per launch, mean over one step: 1.25e+10\n")
    assert bench.profile_traffic("filter_test") == pytest.approx(1.25e10)
    prof.write_text("# x\n\nfilter source sha256[:16]: 0123456789abcdef\n\n"
                    "dram bytes per launch, mean over one step: 1.25e+10\n")
    assert bench.profile_traffic("filter_test") is None
    assert bench.profile_traffic("no_such_profile") is None


def test_committed_profiles_match_the_filter_source():
    # the committed DRAM summaries were taken on the filter code as it stands
    assert bench.profile_traffic("filter_10m_b128") is not None
    assert bench.profile_traffic("filter_1m_b64") is not None
