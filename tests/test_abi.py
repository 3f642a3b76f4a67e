"""The C-ABI library builds, loads, and exports every entry point that
include/*.h declares; argument checks that precede any CUDA call are
exercised without a GPU (CPU only)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21674_gb300 import build
    path = build.build()
    import paper_2511_21674_gb300 as ep
    return ep.load_library(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(eprop_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("eprop_create_network", "eprop_set_inputs_targets", "eprop_simulate",
                     "eprop_read_weights_grads", "eprop_readout", "eprop_sync", "eprop_destroy",
                     "eprop_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_config_struct_layout_matches_header(lib):
    import paper_2511_21674_gb300 as ep
    text = open(os.path.join(ROOT, "include", "eprop.h")).read()
    body = text[text.index("typedef struct eprop_config"):text.index("} eprop_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for line in body.splitlines()[1:]:
        line = line.strip().rstrip(";")
        if not line:
            continue
        typ, rest = line.split(None, 1)
        for name in rest.split(","):
            fields.append(re.sub(r"\[.*\]", "", name.strip()))
    assert [f for f, _ in ep.Config._fields_] == fields


def _cfg(**kw):
    import paper_2511_21674_gb300 as ep
    from workloads import configs as C
    spec = C.Spec(name="t", n_in=2, n_rec=3, n_out=1)
    c = ep.make_config(spec)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _create(lib, cfg, n_src=5, nnz=0):
    import paper_2511_21674_gb300 as ep
    ptr = np.zeros(n_src + 1, np.int64)
    syn = ep.Synapses(n_src=n_src, nnz=nnz, row_ptr=ptr.ctypes.data, target=None, weight=None, delay=None)
    w_out = np.zeros(3, np.float32)
    out = ctypes.c_void_p()
    st = lib.eprop_create_network(ctypes.byref(cfg), ctypes.byref(syn), w_out.ctypes.data, None,
                                  None, 0, None, ctypes.byref(out))
    return st, out, lib.eprop_last_error(None).decode()


@pytest.mark.parametrize("kw,msg", [
    (dict(abi_version=99), "abi_version"),
    (dict(max_delay=0), "max_delay"),
    (dict(max_delay=9), "max_delay"),
    (dict(n_out=0), "sizes"),
    (dict(batch=2, continuous=1), "batch > 1"),
    (dict(feedback=1), "feedback"),
    (dict(trace_kernel=2, update_interval=10), "batched trace kernel"),
    (dict(trace_kernel=5), "trace_kernel must be 0..4"),
    (dict(trace_kernel=4), "trace_kernel 4"),
    (dict(trace_kernel=4, update_interval=10, optimizer=1), "trace_kernel 4"),
    (dict(tau_m=0.0), "time constants"),
])
def test_invalid_config_is_rejected_before_any_cuda_call(lib, kw, msg):
    st, out, err = _create(lib, _cfg(**kw))
    assert st == 1 and not out.value
    assert msg in err


def test_decreasing_drive_table_is_rejected(lib):
    c = _cfg(drive_weight=0.1, n_drive_thr=3)
    c.drive_thr[0], c.drive_thr[1], c.drive_thr[2] = 100, 50, 200
    st, out, err = _create(lib, c)
    assert st == 1 and not out.value
    assert "non-decreasing" in err


def test_inconsistent_synapse_arrays_rejected(lib):
    st, out, err = _create(lib, _cfg(), n_src=7)
    assert st == 1 and "synapse arrays" in err


def test_null_network_calls(lib):
    assert lib.eprop_simulate(None, 10, None) == 1
    assert lib.eprop_sync(None) == 1
    lib.eprop_destroy(None)


def test_autotune_needs_a_network(lib):
    import paper_2511_21674_gb300 as ep
    r = ep.TuneResult()
    assert lib.eprop_autotune(None, ctypes.byref(r)) == 1
