"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/hea.h declares,
and its host-side validation rejects bad arguments before any launch (no GPU needed)."""
import ctypes

import numpy as np
import pytest

from paper_2411_18906_gb300 import build as hbuild
from paper_2411_18906_gb300 import hea


@pytest.fixture(scope="module")
def L():
    hbuild.build()
    return hea.lib()


def test_exports_every_declared_symbol(L):
    names = hea.declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_lattice_handle_host_only(L):
    for kind, dims, M, N, Z in [(hea.HEA_FCC, (40, 40, 40), 3, 256000, [12, 6, 24]),
                                (hea.HEA_BCC, (20, 20, 20), 2, 16000, [8, 6]),
                                (hea.HEA_FCC, (2, 3, 4), 5, 96, [12, 6, 24, 12, 24]),
                                (hea.HEA_BCC, (3, 2, 2), 5, 24, [8, 6, 12, 24, 8])]:
        lat = hea.hea_build_lattice(kind, *dims, M)
        assert lat.N == N
        assert [lat.shell_size(k) for k in range(1, M + 1)] == Z
        assert lat.shell_size(0) == 0 and lat.shell_size(M + 1) == 0


@pytest.mark.parametrize("args", [(2, 4, 4, 4, 3), (0, 1, 4, 4, 3), (0, 4, 4, 4, 0), (1, 4, 4, 4, 6),
                                  (0, 1024, 1024, 1024, 1)])
def test_build_lattice_rejects(L, args):
    h = ctypes.c_void_p()
    assert L.hea_build_lattice(*args, ctypes.byref(h)) == hea.HEA_EINVAL
    assert L.hea_last_error()


def _status(fn, *a):
    try:
        fn(*a)
    except hea.HeaError as e:
        return e.status
    return hea.HEA_OK


class FakePtr:
    """A non-null stand-in pointer: validation must fail before anything dereferences it."""

    def data_ptr(self):
        return 0x1000


def test_validation_before_launch(L):
    lat = hea.hea_build_lattice(hea.HEA_FCC, 4, 4, 4, 3)
    buf = FakePtr()
    # Composition that does not sum to N.
    assert _status(hea.hea_init_config, lat, [10, 10], 1, buf, 0) == hea.HEA_EINVAL
    assert _status(hea.hea_init_config, lat, [300, -44], 1, buf, 0) == hea.HEA_EINVAL
    assert _status(hea.hea_sro_counts, lat, 1, buf, 9, buf, 0) == hea.HEA_EINVAL
    assert _status(hea.hea_sro_counts, lat, 0, buf, 4, buf, 0) == hea.HEA_EINVAL
    good = hea.Objective([64, 64, 64, 64], np.ones(3), np.zeros((3, 4, 4)))
    bad_w = hea.Objective([64, 64, 64, 64], [1.0, -1.0, 1.0], np.zeros((3, 4, 4)))
    bad_n = hea.Objective([0, 64, 64, 128], np.ones(3), np.zeros((3, 4, 4)))
    bad_t = hea.Objective([64, 64, 64, 64], np.ones(3), np.full((3, 4, 4), np.nan))
    bad_m = hea.Objective([64, 64, 64, 64], np.ones(2), np.zeros((2, 4, 4)))
    for obj in (bad_w, bad_n, bad_t, bad_m):
        assert _status(hea.hea_delta_swap, lat, obj, buf, buf, buf, 4, buf, None, 0) == hea.HEA_EINVAL
        assert _status(hea.hea_search, lat, obj, hea.search_params(8, 10), buf, buf, buf, 0) == hea.HEA_EINVAL
    for p in (hea.search_params(0, 10), hea.search_params(5000, 10), hea.search_params(8, -1),
              hea.search_params(8, 10, accept_mode=2), hea.search_params(8, 10, threshold=-1.0),
              hea.search_params(8, 2**32, step0=1), hea.search_params(8, 10, depth_limit=-1)):
        assert _status(hea.hea_search, lat, good, p, buf, buf, buf, 0) == hea.HEA_EINVAL
    assert _status(hea.hea_delta_swap, lat, good, buf, buf, buf, 0, buf, None, 0) == hea.HEA_EINVAL


def test_search_rejects_cells_beyond_shared_memory(L):
    # 5 species need 4 bits per site: 500,000 sites take 250,000 bytes, beyond one CTA's shared memory
    lat = hea.hea_build_lattice(hea.HEA_FCC, 50, 50, 50, 3)
    N = lat.N
    obj = hea.Objective([N // 5] * 5, np.ones(3), np.zeros((3, 5, 5)))
    assert _status(hea.hea_search, lat, obj, hea.search_params(256, 10), FakePtr(), FakePtr(), FakePtr(), 0) \
        == hea.HEA_ENOMEM
    # 4 species fit 2 bits per site, up to about 900,000 sites; 953,312 do not fit
    lat = hea.hea_build_lattice(hea.HEA_FCC, 62, 62, 62, 3)
    N = lat.N
    obj = hea.Objective([N // 4] * 4, np.ones(3), np.zeros((3, 4, 4)))
    assert _status(hea.hea_search, lat, obj, hea.search_params(256, 10), FakePtr(), FakePtr(), FakePtr(), 0) \
        == hea.HEA_ENOMEM


def test_batch_plan_layout(L):
    assert hea.hea_search_batch_plan_bytes(0) == 0
    assert hea.hea_search_batch_plan_bytes(3) > hea.hea_search_batch_plan_bytes(2) > 0
