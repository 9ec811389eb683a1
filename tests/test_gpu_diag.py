"""The library's diagnostics on the GPU: the bounded device-side wait gives up
and reports, and the FP32 FMA throughput the plain path is measured against.

The wait test makes a wait run out without faulting anything: one warp waits
on an mbarrier that no thread arrives at, with a short limit. The kernel must
return on its own, gnn_check must report GNN_ETIMEOUT once, and the context
must stay usable for a following layer call."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as syn
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn
from paper_2410_01657_gb300.graph import MeshGraph

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _small_layer_forward():
    H = 32
    part = MeshGraph((3, 3, 3), 2).partition(2, "slab")
    G = part.to_device(DEV)
    params = syn.gnn_params(5, H, 2, 1)
    layer = gnn.ConsistentGNN(params, precision="bf16", device=DEV).layers[0]
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, layer.edge.tensors() + layer.node.tensors())
    x = torch.randn(part.n_rows, H, device=DEV)
    e = torch.randn(part.n_edges, H, device=DEV).to(torch.bfloat16)
    xo, eo, a = torch.empty_like(x), torch.empty_like(e), torch.empty_like(x)
    gnn.gnn_mp_forward(G, gnn.mp_config(H, "bf16"), W, x, e, xo, eo, a)
    return xo


@pytest.mark.parametrize("limit_us", [50, 2000])
def test_bounded_wait_gives_up_and_reports_timeout(limit_us):
    B.call("gnn_check", None)                      # start from a clear error word
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    B.call("gnn_selftest_bounded_wait", C.c_uint64(limit_us * 1000), B.ptr(status), stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize()                       # the kernel has returned by itself
    assert int(status.item()) == 1                 # the wait gave up (2: it completed)
    ms = ev0.elapsed_time(ev1)
    assert limit_us * 1e-3 <= ms < limit_us * 1e-3 + 50.0
    rc = B.load().gnn_check(None)
    assert rc == B.GNN_ETIMEOUT and "timed out" in B.last_error()
    assert B.load().gnn_check(None) == B.GNN_OK    # read once, then cleared
    xo = _small_layer_forward()                    # the context still runs kernels
    B.call("gnn_check", None)
    assert torch.isfinite(xo).all()


def test_bounded_wait_limit_is_validated():
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert B.load().gnn_selftest_bounded_wait(C.c_uint64(10), B.ptr(status), None) == B.GNN_EINVAL
    assert B.load().gnn_selftest_bounded_wait(C.c_uint64(2_000_000_000), B.ptr(status), None) == B.GNN_EINVAL


def test_fp32_fma_peak_is_measured():
    tf, sms = C.c_double(), C.c_int32()
    B.call("gnn_measure_fp32_fma", C.byref(tf), C.byref(sms), None)
    props = torch.cuda.get_device_properties(0)
    assert sms.value == props.multi_processor_count
    # 2 FLOPs x 128 FP32 lanes x SMs x clock: the measurement must land near that
    # product for a clock between 1 and 2.1 GHz (packed FP32 issue could double it)
    per_ghz = 2 * 128 * sms.value * 1e-3
    assert per_ghz * 0.8 < tf.value < per_ghz * 2.1 * 2.2, tf.value
