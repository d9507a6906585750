"""The device stream generator reproduces streams.KronSpec chunk for chunk
(same updates, same order), so GPU-generated benchmark streams have the net
graph the host-side checks use."""
import numpy as np
import pytest

import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("L,slice_log2", [(6, 12), (9, 13), (11, 18)])
def test_device_chunks_equal_host_chunks_small(L, slice_log2):
    spec = S.KronSpec(L=L, seed=31 + L, target_edges=0.4 * (1 << L) * ((1 << L) - 1) / 2, churn=0.15,
                      n_iso=4, slice_log2=slice_log2)
    gen = gz.DeviceKronStream(spec)
    assert gen.n_chunks == spec.n_chunks
    for c in range(spec.n_chunks):
        du, dv = gen.chunk(c)
        hu, hv = spec.chunk(c)
        assert np.array_equal(_host(du), hu) and np.array_equal(_host(dv), hv), c


def test_device_chunks_equal_host_chunks_v2p17():
    spec = S.KronSpec(L=17, seed=5, target_edges=3.3e9, churn=0.1, n_iso=100, slice_log2=22)
    gen = gz.DeviceKronStream(spec)
    for c in (0, 1, 2049, spec.n_chunks - 1):
        du, dv = gen.chunk(c)
        hu, hv = spec.chunk(c)
        assert len(hu) > 0
        assert np.array_equal(_host(du), hu) and np.array_equal(_host(dv), hv), c
