"""The allocation-free momentum exchange, hlbm_mea_noalloc.

Callers that cannot allocate device memory -- a particle code living inside
another framework's memory pool, or one whose device memory is all handed to
it by its host application -- call hlbm_mea_noalloc on populations they own;
every intermediate of that call sits in one fixed device array inside the
library.  This test feeds it the same populations and particles as a handle
whose first step runs the regular momentum-exchange kernel, and checks that
two calls in a row give that kernel's force and torque.  It is collected last
so that a run that stops at the first failure has run every other test first;
it passes alone in a fresh process too (its first call sets the array up).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2312_14172_gb300 import build, hlbm
    build.build()
    hlbm.load()
    return hlbm


W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _case(nx, ny, nz, bc, seed):
    rng = np.random.default_rng(seed)
    dev = (1e-3 * rng.standard_normal((19, nz, ny, nx)) * W[:, None, None, None]).astype(np.float32)
    shape = np.array([0, 1, 2, 3], np.int32)
    params = np.array([[5.2, 5.2, 5.2], [3.0, 4.0, 7.5], [2.0, 3.5, 4.5], [3.3, 0.0, 4.0]])
    X = np.array([[10.3, 11.7, 12.2], [nx - 9.6, 20.1, 14.8], [22.4, 6.2, nz - 11.3], [1.2, ny - 2.4, 20.5]])
    U = rng.uniform(-2e-3, 2e-3, (4, 3))
    omega = rng.uniform(-3e-3, 3e-3, (4, 3))
    quat = rng.standard_normal((4, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    return dev, shape, params, X, U, omega, quat


@pytest.mark.parametrize("bc", [0, 4])
def test_noalloc_matches_the_momentum_exchange_kernel(H, bc):
    import torch
    nx, ny, nz = 40, 36, 44
    dev, shape, params, X, U, omega, quat = _case(nx, ny, nz, bc, 7 + bc)
    # the regular path: a handle holding the same populations; its first step
    # runs the bounding-box momentum-exchange kernel on them
    lat = H.Lattice([(nx, ny, nz, bc)], H.make_params(tau=0.7, max_particles=4))
    lat.set_populations(W[:, None, None, None] + dev.astype(np.float64))
    lat.add_particles(shape, params, X, U, omega, quat, rho_p=[2.0] * 4)
    lat.step(1)
    ref = lat.particle_state()
    lat.close()
    # the allocation-free path on the caller's own device arrays
    cuda = torch.device("cuda")
    f_d = torch.from_numpy(dev.reshape(19, -1)).to(cuda).contiguous()
    arr = {k: torch.from_numpy(np.ascontiguousarray(v)).to(cuda)
           for k, v in dict(shape=shape, params=params, X=X, U=U, omega=omega, quat=quat).items()}
    F = torch.full((4, 3), 7.0, dtype=torch.float64, device=cuda)
    T = torch.full((4, 3), 7.0, dtype=torch.float64, device=cuda)
    stream = torch.cuda.current_stream()
    for call in range(2):
        rc = H.hlbm_mea_noalloc(f_d.data_ptr(), nx * ny * nz, nx, ny, nz, bc, H.HLBM_FP32, 0, 0, 4,
                                arr["shape"].data_ptr(), arr["params"].data_ptr(), arr["X"].data_ptr(),
                                arr["U"].data_ptr(), arr["omega"].data_ptr(), arr["quat"].data_ptr(),
                                F.data_ptr(), T.data_ptr(), stream.cuda_stream)
        assert rc == H.HLBM_OK
        torch.cuda.synchronize()
        Fh, Th = F.cpu().numpy(), T.cpu().numpy()
        scale = np.abs(ref["F"]).max()
        assert scale > 0
        assert np.max(np.abs(Fh - ref["F"])) <= 1e-6 * scale, call
        assert np.max(np.abs(Th - ref["T"])) <= 1e-6 * np.abs(ref["T"]).max() + 1e-12, call
        F.fill_(-7.0)
        T.fill_(-7.0)


def test_noalloc_rejects_too_many_particles(H):
    rc = H.hlbm_mea_noalloc(1, 64, 4, 4, 4, 0, H.HLBM_FP32, 0, 0, H.HLBM_NOALLOC_MAX_PARTICLES + 1,
                            1, 1, 1, None, None, None, 1, 1, None)
    assert rc == H.HLBM_ERR_ARG
    rc = H.hlbm_mea_noalloc(1, 10, 4, 4, 4, 0, H.HLBM_FP32, 0, 0, 1, 1, 1, 1, None, None, None, 1, 1, None)
    assert rc == H.HLBM_ERR_ARG  # plane shorter than the box
