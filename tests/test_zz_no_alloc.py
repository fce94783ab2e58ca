"""The allocation-free force entry point agrees with the regular one (needs a GB300).

css_compute_forces_noalloc serves callers that cannot allocate device memory where they
evaluate forces; it keeps its scratch in one fixed device array.  It is called here
through the C ABI on device buffers, twice in a row (the second call reuses the array
the first one left behind), and compared with css_compute_forces within the FP64
parity tolerance used by the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests._common import FP64_RTOL

css = pytest.importorskip("paper_2404_19751_gb300")
torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc_fn():
    fn = css.load().css_compute_forces_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                   C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def test_noalloc_forces_match_regular_entry_point():
    fn = _noalloc_fn()
    ctx = css.create(0)
    cfg = synth.make_config("ico5_n1024")
    m, face, bary, r_c = cfg["mesh"], cfg["face"], cfg["bary"], cfg["r_c"]
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    pot = css.Potential(css.POT_HARMONIC, 1.0, r_c, r_c, 1.0)
    n = len(face)
    dface = torch.from_numpy(np.ascontiguousarray(face, np.int32)).cuda()
    dbary = torch.from_numpy(np.ascontiguousarray(bary)).cuda()
    stream = torch.cuda.current_stream()
    for prec in (css.FP64, css.FP32):
        F_ref, E_ref = css.compute_forces(parts, pot, r_c, prec)
        scale = np.max(np.abs(F_ref))
        for call in range(2):
            F = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
            E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = fn(mesh.h, n, dface.data_ptr(), dbary.data_ptr(), C.byref(pot), r_c, prec, F.data_ptr(),
                    E.data_ptr(), stream.cuda_stream)
            assert rc == 0, css.load().css_last_error(ctx.h)
            torch.cuda.synchronize()
            Fh = F.cpu().numpy()
            assert np.isfinite(Fh).all()
            assert np.max(np.abs(Fh - F_ref)) <= FP64_RTOL * scale, (prec, call)
            assert E.item() == pytest.approx(E_ref, rel=1e-10)
    parts.free()
    mesh.free()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _noalloc_fn()
    ctx = css.create(0)
    m = synth.icosphere(2, 1.0)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    pot = css.Potential(css.POT_HARMONIC, 1.0, 0.1, 0.1, 1.0)
    big = 1 << 19   # more particles than the fixed scratch holds: rejected before any access
    dface = torch.zeros(big, dtype=torch.int32, device="cuda")
    dbary = torch.full((big, 3), 1.0 / 3.0, dtype=torch.float64, device="cuda")
    F = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
    rc = fn(mesh.h, big, dface.data_ptr(), dbary.data_ptr(), C.byref(pot), 0.1, css.FP64, F.data_ptr(),
            None, None)
    assert rc == -5
    assert "particles" in css.load().css_last_error(ctx.h).decode()
    mesh.free()
    ctx.close()


def test_noalloc_checks_particle_arrays_on_the_device():
    """A face index equal to nf, or a barycentric triple that does not sum to 1, is caught by
    the device check that runs before any kernel indexes with the caller's arrays; the call
    returns CSS_ERR_INVALID_ARG and a correct call right after still matches css_compute_forces."""
    fn = _noalloc_fn()
    ctx = css.create(0)
    m = synth.icosphere(3, 1.0, noise=0.01, seed=2)
    face, bary = synth.place_uniform(m, 200, 5)
    r_c = 0.3
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    pot = css.Potential(css.POT_HARMONIC, 1.0, r_c, r_c, 1.0)
    n = len(face)
    stream = torch.cuda.current_stream()
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    good_f = np.ascontiguousarray(face, np.int32)
    good_b = np.ascontiguousarray(bary)
    bad_face = good_f.copy()
    bad_face[n // 2] = m.nf                      # one past the last face
    bad_bary = good_b.copy()
    bad_bary[7] = [0.5, 0.5, 0.5]                # sums to 1.5
    nan_bary = good_b.copy()
    nan_bary[3, 1] = float("nan")
    for f_h, b_h in ((bad_face, good_b), (good_f, bad_bary), (good_f, nan_bary)):
        dface = torch.from_numpy(f_h).cuda()
        dbary = torch.from_numpy(b_h).cuda()
        rc = fn(mesh.h, n, dface.data_ptr(), dbary.data_ptr(), C.byref(pot), r_c, css.FP64, F.data_ptr(), None,
                stream.cuda_stream)
        assert rc == -1, rc
        assert "face index" in css.load().css_last_error(ctx.h).decode()
    dface = torch.from_numpy(good_f).cuda()
    dbary = torch.from_numpy(good_b).cuda()
    F_ref, _ = css.compute_forces(parts, pot, r_c, css.FP64)
    rc = fn(mesh.h, n, dface.data_ptr(), dbary.data_ptr(), C.byref(pot), r_c, css.FP64, F.data_ptr(), None,
            stream.cuda_stream)
    assert rc == 0, css.load().css_last_error(ctx.h)
    torch.cuda.synchronize()
    assert np.max(np.abs(F.cpu().numpy() - F_ref)) <= FP64_RTOL * np.max(np.abs(F_ref))
    parts.free()
    mesh.free()
    ctx.close()
