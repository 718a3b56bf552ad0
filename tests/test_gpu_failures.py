"""Failure paths on the device, made without a GPU fault: a clustering
launch whose wait limit is set to zero gives up at its first wait that has
to wait at all, records HDF_ETIMEOUT in the device status word and returns
(the handle reports it; a fresh handle then clusters normally), and an
hdf_create far beyond the device's memory reports HDF_ENOMEM with nothing
left allocated."""
import numpy as np
import pytest
import torch

from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import _lib, api
    return _lib, api


def test_cluster_wait_limit_reports_timeout_and_a_fresh_handle_works(mods):
    L, api = mods
    f_np = synthetic.color_rectangles(256, 256, seed=0)
    f = torch.from_numpy(f_np).cuda()
    flt = api.HDFilter(256, 256, 3, 3, 8, 3.0, 0.2)
    flt.set_wait_limit(0.0)
    flt.cluster(f)
    with pytest.raises(L.HDFError) as e:
        flt.stats()
    assert e.value.code == L.HDF_ETIMEOUT
    flt.close()
    # the context stays usable: a fresh handle clusters as the oracle does
    fresh = api.HDFilter(256, 256, 3, 3, 8, 3.0, 0.2)
    fresh.cluster(f)
    st = fresh.stats()
    assert st["device_error"] == L.HDF_OK and st["K_eff"] == 8
    omu = O.bisecting_kmeans(f_np.reshape(3, -1).T.astype(np.float64), 8)[0]
    gmu = fresh.get_centers()
    assert float(np.max(np.abs(gmu - omu))) <= 1e-5 * float(np.abs(omu).max())
    fresh.close()


def test_wait_limit_argument_checks(mods):
    L, api = mods
    flt = api.HDFilter(16, 16, 3, 3, 4, 1.0, 0.2)
    for bad in (-1.0, float("nan"), 61.0):
        with pytest.raises(L.HDFError) as e:
            flt.set_wait_limit(bad)
        assert e.value.code == L.HDF_EINVAL
    flt.set_wait_limit(1.0)
    flt.close()


def test_create_beyond_device_memory_reports_enomem(mods):
    L, api = mods
    import ctypes as C
    free0, _ = torch.cuda.mem_get_info()
    # 46000 x 46000 pixels, 256 channels, K = 64: the range maps alone need
    # 64 x 2.1e9 x 4 bytes (0.54 TB), beyond any single GPU
    d = api.make_desc(46000, 46000, 256, 3, 64, 3.0, 0.2)
    h = C.c_void_p()
    assert L.lib().hdf_create(C.byref(h), C.byref(d)) == L.HDF_ENOMEM
    assert not h.value
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= (64 << 20), (free0, free1)   # nothing kept
