"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/nw.h declares (no compute calls here)."""
import ctypes

import numpy as np
import pytest

import paper_2412_21103_gb300 as nw
from paper_2412_21103_gb300 import build as nwbuild


@pytest.fixture(scope="module")
def lib():
    nwbuild.build()
    return nw.load()


def test_header_declares_the_boundary():
    names = nw.exported_symbols()
    for required in ["nw_align", "nw_align_batch", "nw_score_all_pairs", "nw_pack", "nw_ctx_create",
                     "nw_ctx_destroy", "nw_strerror"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in nw.exported_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_host_pack_layout(lib):
    out = nw.nw_pack("ACGTacgtA")
    # base k at bits 2*(k%4) of byte k/4: ACGT -> 0b11100100
    assert out.tolist() == [0b11100100, 0b11100100, 0b00000000]
    codes = np.array([0, 1, 2, 3, 0, 1, 2, 3, 0], np.uint8)
    assert nw.pack_codes(codes).tolist() == out.tolist()


def test_host_pack_codes_rejects_code_above_3(lib):
    with pytest.raises(nw.NWError) as e:
        nw.pack_codes(np.array([0, 1, 4], np.uint8))
    assert e.value.status == nw.NW_ERR_BAD_BASE


def test_pool_layout_by_hand(lib):
    """Three sequences of 0, 5 and 70 bases: each starts on a 16-byte
    boundary and takes at least 16 bytes (ceil(70/4) = 18 -> 32 bytes); the
    5-base one ACGTA packs to bytes 0b11100100 (ACGT) and 0b00000000 (A)."""
    seqs = [np.zeros(0, np.uint8), np.array([0, 1, 2, 3, 0], np.uint8), np.full(70, 3, np.uint8)]
    pool, off, lens = nw.pool_of(seqs)
    assert off.tolist() == [0, 16, 32] and lens.tolist() == [0, 5, 70] and pool.size == 64
    assert pool[16:18].tolist() == [0b11100100, 0]
    assert pool[32:49].tolist() == [0xFF] * 17 and pool[49] == 0b00001111   # 70 = 17*4 + 2 bases of T


def test_host_pack_rejects_bad_base(lib):
    with pytest.raises(nw.NWError) as e:
        nw.nw_pack("ACGN")
    assert e.value.status == nw.NW_ERR_BAD_BASE


def test_strerror_and_bound(lib):
    assert lib.nw_strerror(nw.NW_ERR_TIMEOUT) == b"device-side wait timed out"
    assert nw.nw_cigar_bound(3, 4) == 15


def test_context_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert lib.nw_ctx_create(0, None, 0) in (None, 0)


def test_plain_c_program_uses_the_abi(lib, tmp_path):
    """nw.h compiles as C99 (no C++ or torch types at the boundary) and a C
    program linked against libnw.so gets the same answers as the binding."""
    import os
    import shutil
    import subprocess
    import oracle
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = nw.lib_path()
    exe = tmp_path / "c_abi_check"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c_abi_check.c"), so, f"-Wl,-rpath,{os.path.dirname(so)}",
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split(maxsplit=10)
    packed = nw.nw_pack("ACGTacgtA").tolist()
    assert out[0] == "0" and [int(x) for x in out[1:4]] == packed
    assert int(out[4]) == nw.NW_ERR_BAD_BASE
    assert out[5] == "1" and int(out[6]) == oracle.exit_bound(100, 120, 5)
    assert int(out[7]) == nw.nw_cigar_bound(3, 4)
    assert int(out[8]) == int(nw.nw_band_certifies(1000, 1000, 64, 900, True))
    assert int(out[9]) == nw.nw_band_next_width(1000, 1000, 64, 500, True)
    assert out[10].strip() == load_strerror(nw.NW_ERR_BAD_BASE)


def load_strerror(code: int) -> str:
    return nw.load().nw_strerror(code).decode()


def test_checked_build_exports_the_same_boundary():
    """The bounds-checked debug build (-DNW_CHECKS, selected with NW_CHECKS=1)
    compiles and exports every symbol the header declares."""
    path = nwbuild.build(checks=True)
    checked = ctypes.CDLL(path)
    missing = [s for s in nw.exported_symbols() if not hasattr(checked, s)]
    assert not missing, missing
    assert checked.nw_strerror is not None
