"""The allocation-free SR force entry point, vmc_sr_force_static.

It serves callers that cannot let the library allocate device memory (their
memory is owned by another allocator, or they cannot afford the device
synchronisation cudaMalloc/cudaFree may cause).  Here it is called through
the C ABI on device buffers the test owns, and its output is checked against
the context entry point vmc_get_sr_matrices (same samples, FP32 storage) on
two calls in a row, with the tolerance the other SR parity tests use.  This
file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_force_static_matches_context_entry_point():
    torch = pytest.importorskip("torch")
    from paper_1711_11418_gb300 import build, vmc
    from paper_1711_11418_gb300 import inputs as I
    build.build()
    L = vmc.load()
    base = I.ring8_hubbard()
    rows, n_f = 5000, 281                 # 3 row chunks (the last one ragged)
    p = base.copy_with(n_f=n_f, f_idx=np.arange(64, dtype=np.int32), f_sign=np.ones(64, np.int8),
                       params=np.concatenate([base.params[:3],
                                              np.random.default_rng(1).uniform(-1, 1, n_f)]))
    Np = p.Np
    E, O = I.random_samples(rows, Np, seed=21)
    O[:, :40] += 0.3
    W = 50
    with vmc.Context(p, W, seed=1, precision=vmc.MIXED, max_samples=rows // W) as ctx:
        ctx.set_samples(E, O)
        _, g_ref = ctx.get_sr_matrices(with_S=False)
    O32 = torch.tensor(O.astype(np.float32), device="cuda")
    Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    for call in range(2):
        obar = torch.full((Np,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((Np,), float("nan"), dtype=torch.float64, device="cuda")
        ebar = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.vmc_sr_force_static(ptr(O32), Np, rows, Np, ptr(Ed), ptr(obar), ptr(g), ptr(ebar), None)
        torch.cuda.synchronize()
        assert rc == 0, (call, rc)
        g_np = g.cpu().numpy()
        assert np.max(np.abs(g_np - g_ref)) <= 1e-10 * np.max(np.abs(g_ref)), call
        o_ref = O.astype(np.float32).astype(np.float64).mean(axis=0)
        assert np.max(np.abs(obar.cpu().numpy() - o_ref)) <= 1e-10 * np.max(np.abs(o_ref)), call
        assert ebar.item() == pytest.approx(E.mean(), rel=1e-12), call
    # Beyond the static scratch: rejected before anything is launched.  One
    # row of Np = 2^20 + 1 parameters needs 2^20 + 1 scratch doubles; every
    # buffer passed is large enough for the arguments, so a regression of the
    # guard could not read or write outside them.
    Nbig = vmc.FORCE_STATIC_MAX_DOUBLES + 1
    Obig = torch.zeros(Nbig, dtype=torch.float32, device="cuda")
    ob = torch.zeros(Nbig, dtype=torch.float64, device="cuda")
    gb = torch.zeros(Nbig, dtype=torch.float64, device="cuda")
    rc = L.vmc_sr_force_static(ptr(Obig), Nbig, 1, Nbig, ptr(Ed), ptr(ob), ptr(gb), ptr(ebar), None)
    assert rc == -1
    torch.cuda.synchronize()
    assert float(ob.abs().max()) == 0.0 and float(gb.abs().max()) == 0.0


def test_force_static_more_row_chunks_than_grid_rows():
    """65,536 chunks of 2048 rows (one parameter): more chunks than a grid
    has rows in y, taken by a loop inside the kernel."""
    torch = pytest.importorskip("torch")
    from paper_1711_11418_gb300 import build, vmc
    build.build()
    L = vmc.load()
    rows = 65535 * 2048 + 5
    gen = torch.Generator(device="cuda").manual_seed(3)
    O = torch.rand(rows, dtype=torch.float32, device="cuda", generator=gen)
    # E correlated with O, so that g (about var O = 1/12) is far from zero
    E = O.double() + 0.5 * torch.rand(rows, dtype=torch.float64, device="cuda", generator=gen)
    obar = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    ebar = torch.zeros(1, dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = L.vmc_sr_force_static(ptr(O), 1, rows, 1, ptr(E), ptr(obar), ptr(g), ptr(ebar), None)
    torch.cuda.synchronize()
    assert rc == 0
    O64 = O.double()
    o_ref = O64.mean()
    g_ref = ((O64 - o_ref) * (E - E.mean())).mean()
    assert abs(obar.item() - o_ref.item()) <= 1e-12 * abs(o_ref.item())
    assert abs(ebar.item() - E.mean().item()) <= 1e-12 * abs(E.mean().item())
    assert abs(g.item() - g_ref.item()) <= 1e-10 * abs(g_ref.item())
