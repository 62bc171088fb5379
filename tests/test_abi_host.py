"""The C-ABI library builds, loads and exports every declared symbol; host-side validation (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_06634_gb300 import _native, build
    build.build()
    return _native.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "bioem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bioem_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1609_06634_gb300 import _native
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, f"{name} has no ctypes signature"


def test_host_side_validation(lib):
    assert lib.bioem_status_string(0) == b"ok"
    assert lib.bioem_status_string(-6) == b"numerically degenerate input"
    assert lib.bioem_last_error(None) == b"null context"
    assert lib.bioem_create(None, 0, None) == -1
    assert lib.bioem_images_count(None) == -1
    assert lib.bioem_projset_count(None) == -1
    lib.bioem_free_images(None)
    lib.bioem_free_projset(None)
    assert lib.bioem_prepare_images(None, None, 1, 32, 32, 1.0, None) == -1
    assert lib.bioem_score(None, None, None, 0, None, None) == -1
    assert lib.bioem_get_status(None, None) == -1
    assert lib.bioem_set_scratch_limit(None, 1 << 20) == -1


def test_package_has_no_cpu_path():
    import paper_1609_06634_gb300 as pkg
    src = open(pkg.__file__).read()
    assert "oracle" not in src.replace("no CPU path", "")
    assert "import numpy" in src   # host-side marshalling of CTF rows only


def test_timing_hook_names_match_the_header():
    """The kernel names bioem_kernel_time accepts (the library's table) are the ones the header lists."""
    src = open(os.path.join(ROOT, "paper_1609_06634_gb300", "csrc", "abi.cu")).read()
    table = re.search(r"bioem_kernel_names\[KID_COUNT\]\s*=\s*\{(.*?)\};", src, flags=re.S).group(1)
    accepted = set(re.findall(r'"(k_[a-z_]+)"', table))
    hdr = open(os.path.join(ROOT, "include", "bioem.h")).read()
    doc = re.search(r"bioem_kernel_time synchronises(.*?)\*/", hdr, flags=re.S).group(1)
    documented = set(re.findall(r'"(k_[a-z_]+)"', doc))
    assert accepted and accepted == documented, (accepted ^ documented)


def test_autotune_cache_rejects_corrupted_entries(lib, tmp_path):
    """Entries for unsupported sizes, windows beyond an instance, chunks that are not whole batches
    (pairs per batch: 15 / 10 / 7 / 2 at 64 / 96 / 128 / 192 px) or out of range, and malformed
    lines are skipped; valid ones are taken."""
    import paper_1609_06634_gb300 as bioem
    path = tmp_path / "tune.txt"
    path.write_text("128 16 224\n"        # valid: 32 batches of 7
                    "64 8 120\n"          # valid
                    "128 16 5\n"          # not a multiple of 7
                    "999 4 64\n"          # unsupported size
                    "128 99 70\n"         # window beyond the 128 px instance
                    "192 24 0\n"          # empty chunk
                    "96 12 8000\n"        # above 4096
                    "64 -1 30\n"          # negative window
                    "garbage line\n"
                    "128 4\n"             # too few fields
                    "128 4 70 extra\n"    # trailing token
                    "\n")
    assert bioem.autotune_load(str(path)) == (2, 9)
    with pytest.raises(bioem.BioEMError):
        bioem.autotune_load(str(tmp_path / "missing.txt"))
    assert lib.bioem_autotune_load(None, None, None) == -1
