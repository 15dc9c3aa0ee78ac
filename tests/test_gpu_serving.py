"""The serving loop on the device: every request completes, and each
request's result is the same whether it ran in a mix of many domains or
alone."""
import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm
from paper_1503_03337_gb300.serving import BatchBackend, SequentialBackend, Server, summarize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()
    return torch


def trace():
    return inputs.request_trace(14, rate=2000.0, seed=3, lmin=16, lmax=40, max_steps=300)


def serve(torch, backend):
    srv = Server(backend, check_every=100, tol=1e-8, chunk=25, keep_fields=True)
    t = trace()
    out = srv.run(t)
    torch.cuda.synchronize()
    backend.close()
    return out


def test_results_same_in_mix_and_alone(torch):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        mixed = serve(torch, BatchBackend(16, 0, stream.cuda_stream))
        alone = serve(torch, BatchBackend(1, 0, stream.cuda_stream))
    assert len(mixed) == len(alone) == 14
    for rid in mixed:
        assert mixed[rid].steps == alone[rid].steps
        assert mixed[rid].fingerprint == alone[rid].fingerprint, rid
        # the whole velocity field, bit for bit
        assert mixed[rid].u is not None and np.array_equal(mixed[rid].u, alone[rid].u), rid
    s = summarize(mixed, max(o.done for o in mixed.values()))
    assert s["glups"] > 0 and s["p99_s"] >= s["p50_s"]


def test_sequential_backend_matches_for_steady_drives(torch):
    """Cavity and duct requests (no time-dependent force) give the same
    result through single-domain handles as through the batch."""
    stream = torch.cuda.Stream()
    keep = [r for r in trace() if r.kind != "pulsatile"]
    with torch.cuda.stream(stream):
        a = Server(BatchBackend(16, 0, stream.cuda_stream), check_every=100, chunk=25,
                   keep_fields=True).run(keep)
        b = Server(SequentialBackend(stream.cuda_stream), check_every=100, chunk=25,
                   keep_fields=True).run(keep)
    torch.cuda.synchronize()
    for r in keep:
        assert a[r.rid].fingerprint == b[r.rid].fingerprint
        assert np.array_equal(a[r.rid].u, b[r.rid].u), r.rid
        assert a[r.rid].residual == b[r.rid].residual
