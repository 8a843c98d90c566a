"""The in-tree build notices every source the library is compiled from: a
kernel body in a .cuh header that is newer than the library makes it stale,
so a test run never exercises an old binary. The check moves only the
modification time of a stand-in library file, never of a source."""
import glob
import os

from paper_1912_04379_gb300 import build


def test_every_cuh_header_is_a_dependency():
    cuh = glob.glob(os.path.join(build.CSRC, "*.cuh"))
    assert cuh, "no .cuh kernel headers found"
    deps = set(build._deps())
    for f in cuh:
        assert f in deps, f"{os.path.basename(f)} is not watched by the build"


def test_newer_cuh_marks_the_library_stale(tmp_path):
    lib = tmp_path / "libstandin.so"
    lib.write_bytes(b"")
    newest = max(os.path.getmtime(d) for d in build._deps())
    os.utime(lib, (newest + 10, newest + 10))
    assert build.up_to_date(str(lib))
    for f in glob.glob(os.path.join(build.CSRC, "*.cuh")):
        t = os.path.getmtime(f)
        os.utime(lib, (t - 10, t - 10))          # the header is now newer than the library
        assert not build.up_to_date(str(lib)), f"{os.path.basename(f)} change not seen"
        os.utime(lib, (newest + 10, newest + 10))
