"""GPU serving: every result is the same alone and in the mix; the loop completes a Poisson
request stream with mixed N."""
import numpy as np
import pytest
import torch

from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu


def _server(**kw):
    from paper_2509_01855_gb300.serve import Server
    return Server(**kw)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_same_alone_and_in_the_mix(dtype):
    reqs = [dict(id=i, arrival=0.0, N=n, rf=rf, tf=tf, keep=True)
            for i, (n, rf, tf) in enumerate([(256, 1.3, 12.0), (1024, 1.8, 25.0), (512, 1.5, 20.0),
                                             (4096, 1.2, 10.0), (256, 2.0, 30.0), (2048, 1.6, 17.0)])]
    alone = _server(max_slots=1, dtype=dtype)
    res_alone, _ = alone.run(reqs, realtime=False)
    alone.close()
    mix = _server(max_slots=6, dtype=dtype)
    res_mix, stats = mix.run(reqs, realtime=False)
    mix.close()
    for a, b in zip(res_alone, res_mix):
        assert a["status"] == "ok" and b["status"] == "ok", (a, b)
        assert np.array_equal(a["solution"], b["solution"])     # bitwise
        assert a["newton_iterations"] == b["newton_iterations"]
    assert stats["solved"] == len(reqs)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_poisson_stream_mixed_N(dtype):
    reqs = synth.serving_requests(48, rate=200.0, kmin=8, kmax=13)
    srv = _server(max_slots=8, dtype=dtype)
    res, st = srv.run(reqs, realtime=True)
    srv.close()
    assert st["solved"] == 48, [r for r in res if r["status"] != "ok"][:3]
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert all(r["newton_iterations"] <= 10 for r in res)
