"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/*.h declares (no compute calls: this runs on CPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1302_3876_gb300 import build as libbuild
from paper_1302_3876_gb300 import enkf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"ENKF_API\s+[\w\s\*]+?\b(enkf_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return enkf.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("enkf_ism_plan", "enkf_ism_analysis", "enkf_obs_prep", "enkf_ism_plan_destroy",
                     "enkf_status_string", "enkf_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_exposes_declared_names():
    for name in declared_functions():
        assert hasattr(enkf, name), name


def test_status_strings(lib):
    assert enkf.enkf_status_string(enkf.ENKF_OK) == "ENKF_OK"
    assert enkf.enkf_status_string(enkf.ENKF_ERR_TIMEOUT) == "ENKF_ERR_TIMEOUT"
    assert enkf.enkf_status_string(99) == "ENKF_UNKNOWN_STATUS"


def test_plan_rejects_bad_arguments_before_touching_the_device(lib):
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_plan(10, 0, 4, enkf.ENKF_FP32)
    assert e.value.status == enkf.ENKF_ERR_SHAPE
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_plan(10, 10, 4, 17)
    assert e.value.status == enkf.ENKF_ERR_ARG
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_plan(10, 10, 4, enkf.ENKF_FP32, flags=0x100)
    assert e.value.status == enkf.ENKF_ERR_ARG


def test_library_is_in_tree():
    assert os.path.commonpath([libbuild.LIB_PATH, ROOT]) == ROOT
