"""The in-tree build's dependency tracking (CPU, no compiler run): an object
is rebuilt when its source, a .cu file that source includes, or a header is
newer than it."""
import os

from paper_2105_10312_gb300 import _build as B


def test_capacity_builds_depend_on_the_kernel_source_they_include():
    """The 64- and 256-task builds re-include a kernel source: that source is
    among their dependencies, and every listed source exists."""
    inc = {f: B._included_sources(os.path.join(B.CSRC, f)) for f in B.CU_SOURCES}
    for f, deps in inc.items():
        assert os.path.exists(os.path.join(B.CSRC, f)), f
        for d in deps:
            assert os.path.exists(d), (f, d)
    assert os.path.join(B.CSRC, "k_alloc.cu") in inc["k_alloc_small.cu"]
    assert os.path.join(B.CSRC, "k_alloc.cu") in inc["k_alloc_wide.cu"]
    assert os.path.join(B.CSRC, "k_test.cu") in inc["k_test_wide.cu"]
    assert inc["k_alloc.cu"] == []


def test_an_object_is_stale_when_missing_or_older_than_a_dependency(tmp_path):
    obj, dep = tmp_path / "a.o", tmp_path / "a.cu"
    dep.write_text("x")
    assert B._stale(str(obj), [str(dep)])  # never built
    obj.write_text("y")
    os.utime(obj, (2000, 2000))
    os.utime(dep, (1000, 1000))
    assert not B._stale(str(obj), [str(dep), str(tmp_path / "gone.h")])  # a missing dependency is ignored
    os.utime(dep, (3000, 3000))
    assert B._stale(str(obj), [str(dep)])
