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


class FakeBuf(FakePtr):
    """A stand-in device buffer of a given size (validation reads only its size)."""

    def __init__(self, nbytes, addr=0x100000):
        self.nbytes, self.addr = nbytes, addr

    def data_ptr(self):
        return self.addr

    def numel(self):
        return self.nbytes

    def element_size(self):
        return 1


def test_global_search_validation(L):
    lat = hea.hea_build_lattice(hea.HEA_FCC, 4, 4, 4, 3)
    obj = hea.Objective([64, 64, 64, 64], np.ones(3), np.zeros((3, 4, 4)))
    good = hea.global_params(64, 6, 64, 8)
    need = hea.hea_global_search_workspace_bytes(lat, obj, good)
    # pool of 64 x 256 bytes + counts + F^2 + order + 32... descriptors and results
    assert need >= 64 * 256 + 64 * 48 * 4 + 64 * 8 + 64 * 4
    assert hea.hea_global_search_workspace_bytes(lat, obj, hea.global_params(128, 10, 256, 10)) > need
    bad = [hea.global_params(0, 6, 64, 8), hea.global_params(5000, 6, 64, 8), hea.global_params(64, 0, 64, 8),
           hea.global_params(64, 6, 0, 8), hea.global_params(64, 6, 5000, 8), hea.global_params(64, 6, 64, 0),
           hea.global_params(64, 6, 64, 8, n_refine=65), hea.global_params(64, 6, 64, 8, n_refine=10, n_keep=6),
           hea.global_params(64, 6, 64, 8, max_steps=0), hea.global_params(64, 6, 64, 8, accept_mode=2),
           hea.global_params(64, 70000, 64, 8)]
    b = FakePtr()
    for p in bad:
        assert hea.hea_global_search_workspace_bytes(lat, obj, p) == 0
        assert _status(hea.hea_global_search, lat, obj, p, b, b, b, None, b, FakeBuf(need), 0) == hea.HEA_EINVAL
    # short or misaligned workspace
    assert _status(hea.hea_global_search, lat, obj, good, b, b, b, None, b, FakeBuf(need - 1), 0) == hea.HEA_EINVAL
    assert _status(hea.hea_global_search, lat, obj, good, b, b, b, None, b, FakeBuf(need, 0x100010), 0) == hea.HEA_EINVAL
    bad_n = hea.Objective([0, 64, 64, 128], np.ones(3), np.zeros((3, 4, 4)))
    assert _status(hea.hea_global_search, lat, bad_n, good, b, b, b, None, b, FakeBuf(need), 0) == hea.HEA_EINVAL
    # a cell with `tasks` candidate slots beyond one CTA's shared memory
    big = hea.hea_build_lattice(hea.HEA_FCC, 50, 50, 50, 3)
    obj5 = hea.Objective([big.N // 5] * 5, np.ones(3), np.zeros((3, 5, 5)))
    p = hea.global_params(4, 1, 256, 8)
    assert _status(hea.hea_global_search, big, obj5, p, b, b, b, None, b,
                   FakeBuf(hea.hea_global_search_workspace_bytes(big, obj5, p)), 0) == hea.HEA_ENOMEM
