"""ms_evaluate_noalloc: the allocation-free material evaluation.

Some callers cannot allocate device memory (their memory belongs to another
allocator, or they must not allocate while they run), so this entry point
keeps its scratch in a fixed device array inside the library.  The test calls
it through the C ABI twice in a row and checks its outputs against the
existing entry points that compute the same thing: the mean stress against
ms_run's first material evaluation of a resumed state, and the stress and
internal-variable fields against gsm_update applied phase by phase.  This
file is collected last so that a stop-at-first-failure run has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def soa(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_noalloc_evaluation_matches_existing_entry_points(gsm):
    import torch
    lib = gsm.load()
    N = 16
    nvox = N ** 3
    ph = synth.sphere_phase(N, 0.2)
    phase = torch.from_numpy(ph).cuda()
    laws = [gsm.norton(*synth.MATRIX_16), gsm.elastic(*synth.INCLUSION_16)]
    arr = (ctypes.c_void_p * 2)(*[m.handle.value for m in laws])
    laws_ptr = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
    stream = torch.cuda.current_stream()
    mask = ph.reshape(-1) == 0

    for call, (seed, h) in enumerate([(1, 0.1), (2, 0.01)]):
        eps_np, zn_np = synth.material_batch(nvox, seed=seed, eps_amp=0.01, z_amp=0.002)
        eps, zn = soa(eps_np), soa(zn_np)
        sigma = torch.full((6, nvox), float("nan"), dtype=torch.float64, device="cuda")
        z = torch.full_like(sigma, float("nan"))
        mean = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ms_evaluate_noalloc(N, ctypes.c_void_p(phase.data_ptr()), 2, laws_ptr, ctypes.c_double(h),
                                     ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(zn.data_ptr()),
                                     ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, f"call {call}: rc {rc}"
        torch.cuda.synchronize()
        sig_n, z_n_out, mean_n = sigma.cpu().numpy(), z.cpu().numpy(), mean.cpu().numpy()

        # the existing basic-scheme entry point: one material evaluation of the same state
        E = eps_np.mean(axis=0)
        st_eps, st_z = eps.clone(), zn.clone()
        ctx = gsm.ms_create(phase, laws)
        out = gsm.ms_run(ctx, E[None], [h], forced_iters=[1], eps=st_eps, z=st_z, resume=True, E_prev=E)
        gsm.ms_destroy(ctx)
        assert rel(mean_n, out["Sigma"][0]) < TOL
        z_ms = st_z.cpu().numpy()
        assert rel(z_n_out[:, mask], z_ms[:, mask]) < TOL
        assert np.array_equal(z_n_out[:, ~mask], np.zeros((6, int((~mask).sum()))))

        # the existing material entry point, phase by phase
        for p, m in enumerate(laws):
            sel = np.nonzero(ph.reshape(-1) == p)[0]
            e_p, z_p = soa(eps_np[sel]), soa(zn_np[sel])
            s_p, zz_p = torch.empty_like(e_p), torch.empty_like(e_p)
            gsm.gsm_update(m, e_p, z_p, h, s_p, zz_p)
            torch.cuda.synchronize()
            assert rel(sig_n[:, sel], s_p.cpu().numpy()) < TOL
            if p == 0:
                assert rel(z_n_out[:, sel], zz_p.cpu().numpy()) < TOL
        assert rel(mean_n, sig_n.mean(axis=1)) < TOL


def test_noalloc_rejects_bad_sizes(gsm):
    import torch
    lib = gsm.load()
    laws = [gsm.elastic(70.0, 0.3)]
    arr = (ctypes.c_void_p * 1)(laws[0].handle.value)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    for N in (1, 1025):
        rc = lib.ms_evaluate_noalloc(N, p, 1, ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), ctypes.c_double(0.1),
                                     p, p, p, p, p, None)
        assert rc == gsm.GSM_EINVAL


def test_noalloc_call_allocates_no_device_memory(gsm):
    """After a first call (which sets the device up), a further call leaves the
    device's free memory and torch's reserved pool unchanged."""
    import torch
    lib = gsm.load()
    N = 24
    nvox = N ** 3
    ph = torch.from_numpy(synth.sphere_phase(N, 0.2)).cuda()
    laws = [gsm.norton(*synth.MATRIX_16), gsm.elastic(*synth.INCLUSION_16)]
    arr = (ctypes.c_void_p * 2)(*[m.handle.value for m in laws])
    eps_np, zn_np = synth.material_batch(nvox, seed=4, eps_amp=0.01, z_amp=0.002)
    eps, zn = soa(eps_np), soa(zn_np)
    sigma, z = torch.empty_like(eps), torch.empty_like(eps)
    mean = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        return lib.ms_evaluate_noalloc(N, ctypes.c_void_p(ph.data_ptr()), 2,
                                       ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), ctypes.c_double(0.1),
                                       ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(zn.data_ptr()),
                                       ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                       ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(stream.cuda_stream))

    assert call() == 0
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    first = mean.cpu().numpy()
    assert call() == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert np.array_equal(mean.cpu().numpy(), first)
