"""The C-ABI library builds for sm_103a, loads, and exports every declared
entry point (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1205_1222_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nbreg.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


def test_header_and_binding_agree():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    syms = set(re.findall(r"\s[TW]\s+(\S+)", out))
    missing = [s for s in _declared() if s not in syms]
    assert not missing, missing


def test_library_loads_and_answers_host_queries(lib_path):
    lib = binding.library()
    assert binding.strerror(binding.NB_ERR_TIMEOUT).startswith("a bounded")
    for mode in (binding.NB_FP64, binding.NB_MIXED, binding.NB_FP32):
        n = binding.nb_num_kernel_configs(mode)
        assert n >= 1
        cfgs = [binding.nb_get_kernel_config(mode, i).as_tuple() for i in range(n)]
        assert len(set(cfgs)) == n
        for w, ipw, jt, split, packed in cfgs:
            assert w > 0 and ipw > 0 and jt % 32 == 0 and split == 0
            assert packed in ((0,) if mode == binding.NB_FP64 else (0, 2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13, 14, 20))
    assert lib.nb_create is not None


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_without_a_device_fails_cleanly(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.NbError) as e:
        binding.nb_create(0, 1024)
    assert e.value.status == binding.NB_ERR_ARG


def test_tuned_table_calls_reject_a_null_context(lib_path):
    lib = binding.library()
    t = binding.nb_tuned()
    assert lib.nb_num_tuned(None) == 0
    assert lib.nb_set_tuned(None, ctypes.byref(t)) == binding.NB_ERR_ARG
    assert lib.nb_get_tuned(None, 0, ctypes.byref(t)) == binding.NB_ERR_ARG


def test_tuned_table_file_format_is_checked(tmp_path):
    from paper_1205_1222_gb300 import autotune
    p = tmp_path / "t.json"
    p.write_text('{"format": "something-else", "entries": []}')
    with pytest.raises(ValueError):
        autotune.load(None, str(p))
