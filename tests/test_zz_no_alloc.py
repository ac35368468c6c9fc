"""The allocation-free entry point tdz_cn1d_propagate_noalloc, checked through the C ABI against
the batch entry point (tdz_propagate, binary64) on two calls in a row.

It serves callers that cannot call cudaMalloc (a host framework that owns all device memory in its
own pool, or code that must not risk an implicit device synchronisation); its scratch is a fixed
device array inside the library. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the binary64 parity tolerance used by the 1-D tests


def _entry(tdz):
    f = tdz._lib.tdz_cn1d_propagate_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_double, C.c_int64, C.c_int64, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    return f


# (4098, 8): n = 4096 = TDZ_NOALLOC_MAX_N at the largest degree, the full static scratch;
# (771, 8): n = 3 P 32 + 1, one row past the size where the 32 chunks of the single warp are
# exactly 3P rows long, so the last chunk is ragged
@pytest.mark.parametrize("nspl,p", [(600, 6), (1000, 7), (30, 3), (4098, 8), (771, 8)])
def test_noalloc_matches_batch_entry_two_calls(nspl, p):
    import torch

    import paper_2608_18472_b300 as tdz
    dev = torch.device("cuda:0")
    knots = wl.knots_for_nsplines(-60.0, 60.0, nspl, p)
    med = wl.softcore_medium(2.0)
    ops = tdz.assemble_1d(knots, p, med, p + 1)
    n = ops.n
    _, c0 = ops.ground_state()
    dt, ns = 0.05, 150
    field = wl.sin2_pulse(wl.time_grid(dt, 2 * ns), 0.06, 0.2, 2.0)[:, 0]

    # reference: the batch entry point, two calls
    b = tdz.Batch([ops], [0], tdz.FP64)
    b.set_state(0, c0)
    ref = []
    for call in range(2):
        b.propagate(field[call * ns:(call + 1) * ns + 1].reshape(1, ns + 1, 1), dt, call * ns, ns)
        ref.append((b.get_state(0), b.observe(0)[0].copy()))

    # allocation-free entry point, caller-owned device buffers
    bands = torch.tensor(np.stack([ops.band(k) for k in ("S", "H0", "D", "G", "K")]), dtype=torch.float64, device=dev)
    state = torch.tensor(np.stack([c0.real, c0.imag], axis=1).reshape(-1), dtype=torch.float64, device=dev)
    fdev = torch.tensor(field, dtype=torch.float64, device=dev)
    obs = torch.zeros((ns, 5), dtype=torch.float64, device=dev)
    f = _entry(tdz)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        st = C.c_int(-99)
        rc = f(bands.data_ptr(), n, p, fdev.data_ptr() + 8 * call * ns, dt, call * ns, ns, state.data_ptr(),
               obs.data_ptr(), stream, C.byref(st))
        assert rc == tdz.TDZ_OK, tdz.last_error()
        assert st.value == tdz.TDZ_OK
        torch.cuda.synchronize()
        s = state.cpu().numpy()
        c = s[0::2] + 1j * s[1::2]
        rc_state, rc_obs = ref[call]
        assert np.linalg.norm(c - rc_state) / np.linalg.norm(rc_state) < TOL
        o = obs.cpu().numpy()
        assert np.max(np.abs(o[:, 0] - rc_obs[:, 0])) < 1e-12
        for col in (2, 3, 4):
            assert np.max(np.abs(o[:, col] - rc_obs[:, col])) < TOL * max(1.0, np.max(np.abs(rc_obs[:, col])))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    import paper_2608_18472_b300 as tdz
    f = _entry(tdz)
    dev = torch.device("cuda:0")
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    rc = f(buf.data_ptr(), 5000, 6, buf.data_ptr(), 0.05, 0, 1, buf.data_ptr(), buf.data_ptr(), None, None)
    assert rc == tdz.TDZ_EINVAL
    assert "TDZ_NOALLOC_MAX_N" in tdz.last_error()
