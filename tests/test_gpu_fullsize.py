"""Full-size GPU parity on the five workloads, in the launch configuration the benchmark times.

Every output the oracle can produce within a few minutes over the host cores is compared
element by element (all results are exact integers, the adjoint's float32 is exact too):

- 128^3 voxel volume, d = 256, T = 128: every direction;
- 1024^2 mesh, d = 1024, T = 512, default range: the first and last direction of every
  32-direction tile (the gather works one tile at a time), 64 directions;
- 4096 blob images, d = 64, T = 64: every image of the graph-captured batched launch;
- 256 volumes of 64^3, d = 128, T = 128: the batched forward of two volumes, the target batch of
  the same two, and the autograd gradient of the mean squared error over the whole batch for
  both (all 128 directions against the oracle's exact adjoint); plus central finite differences
  of the GPU forward at h = 1e-3 on tie-free vertices.
- 64^2 image, d = 32, T = 64 and its ECF are covered completely in test_gpu_cubical.py;
- the intensity-filter ECF at the paper's throughput sizes 2048^2 and 128^3, T = 1000 and 10000,
  uniform [0, 1) filters over [0, 1], through the same call the benchmark times.

The oracle runs in spawned worker processes, one per host core; all its work is submitted when
the module starts so that it overlaps the GPU work.
"""
from fractions import Fraction

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch
from oracle_pool import OraclePool, ecf_filter, ecf_grid, images, mesh_dirs, voxel_dirs, volume_adjoint

pytestmark = pytest.mark.gpu

VOL_CHECKED = (17, 200)          # volumes of the differentiation batch compared with the oracle
ECF_CASES = [([2048, 2048], 10000), ([128, 128, 128], 10000), ([2048, 2048], 1000), ([128, 128, 128], 1000)]


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


@pytest.fixture(scope="module")
def jobs(P):
    pool = OraclePool()
    J = {}
    # the longest single tasks first: the T = 10000 ECFs (the oracle counts thresholds one by
    # one), then one volume's transform, target and adjoint each
    J["ecf"] = [pool.submit(ecf_grid, dims, 70 + i, T) for i, (dims, T) in enumerate(ECF_CASES)]
    wv = S.volume_batch_diff()
    from oracle import oracle as O

    N = len(wv.grids) * len(wv.dirs) * wv.T
    J["vol"] = {k: pool.submit(volume_adjoint, O.to_fixed(wv.grids[k], 24), O.to_fixed(wv.target[k], 24), wv.dims,
                               wv.dirs, wv.T, wv.lo, wv.hi, N) for k in VOL_CHECKED}
    del wv
    mesh_idx = sorted({t * 32 for t in range(32)} | {t * 32 + 31 for t in range(32)})
    J["mesh_idx"] = mesh_idx
    J["mesh"] = [pool.submit(mesh_dirs, mesh_idx[i:i + 2]) for i in range(0, len(mesh_idx), 2)]
    J["voxel"] = [pool.submit(voxel_dirs, i, i + 4) for i in range(0, 256, 4)]
    J["images"] = [pool.submit(images, i, i + 64) for i in range(0, 4096, 64)]
    J["pool"] = pool
    yield J
    pool.close()


def test_volumes3d_full_batch_forward_and_adjoint(P, jobs):
    """The batched forward and the autograd gradient of the MSE over all 256 volumes (the
    forward + backward the benchmark times), two volumes against the oracle in every direction."""
    wl = S.volume_batch_diff()
    dirs = cuda(wl.dirs)
    flat = cuda(wl.grids.reshape(-1))
    b = P.CubicalBatch(flat=flat, dims=[wl.dims] * len(wl.grids), frac_bits=24)
    bt = P.CubicalBatch(flat=cuda(wl.target.reshape(-1)), dims=[wl.dims] * len(wl.grids), frac_bits=24)
    B = bt.wect(dirs, wl.T, wl.lo, wl.hi)
    Breal = B.to(torch.float64) * 2.0 ** -24
    w = flat.clone().requires_grad_(True)
    W = P.WECTFunction.apply(b, w, dirs, wl.T, wl.lo, wl.hi)
    loss = ((W - Breal) ** 2).mean()
    loss.backward()
    g = w.grad.detach().cpu().numpy().reshape(len(wl.grids), -1)
    Wfix = (W.detach() * 2.0 ** 24).to(torch.int64).cpu().numpy()
    B = B.cpu().numpy()
    for k in VOL_CHECKED:
        Wk, Bk, gk = jobs["vol"][k].get()
        assert np.array_equal(Wfix[k], Wk), k
        assert np.array_equal(B[k], Bk), k
        assert np.array_equal(g[k], gk), k


def _tie_free(vw, dims, v, k):
    """No vertex sharing a cell with v has a fixed weight within k of v's."""
    n = len(dims)
    idx, r = [], v
    for a in range(n):
        idx.append(r % dims[a])
        r //= dims[a]
    strides = [int(np.prod(dims[:a])) for a in range(n)]
    for off in np.ndindex(*([3] * n)):
        if all(o == 1 for o in off):
            continue
        u = [idx[a] + off[a] - 1 for a in range(n)]
        if any(u[a] < 0 or u[a] >= dims[a] for a in range(n)):
            continue
        if abs(int(vw[sum(u[a] * strides[a] for a in range(n))]) - int(vw[v])) <= k:
            return False
    return True


def test_volumes3d_finite_differences(P):
    """Central finite differences of the GPU forward, h = 1e-3 (2^-24 fixed point: k = 16777
    units, so the step is symmetric and exact), on 24 tie-free vertices of one volume including
    corners and faces, against the GPU autograd gradient of the full-batch MSE.  The loss is
    quadratic in a tie-free weight, so the difference quotient, computed exactly in integers, is
    the derivative itself; the bar is 1e-6 relative."""
    wl = S.volume_batch_diff()
    dirs = cuda(wl.dirs)
    count = len(wl.grids)
    N = count * len(wl.dirs) * wl.T
    b = P.CubicalBatch(flat=cuda(wl.grids.reshape(-1)), dims=[wl.dims] * count, frac_bits=24)
    bt = P.CubicalBatch(flat=cuda(wl.target.reshape(-1)), dims=[wl.dims] * count, frac_bits=24)
    B = bt.wect(dirs, wl.T, wl.lo, wl.hi)
    w = cuda(wl.grids.reshape(-1)).requires_grad_(True)
    W = P.WECTFunction.apply(b, w, dirs, wl.T, wl.lo, wl.hi)
    (((W - B.to(torch.float64) * 2.0 ** -24) ** 2).mean()).backward()
    kv = 5
    g = w.grad.detach().cpu().numpy().reshape(count, -1)[kv]
    Bk = B[kv].cpu().numpy().astype(object)
    vw = np.rint(np.ldexp(wl.grids[kv].astype(np.float64).ravel(), 24)).astype(np.int64)
    k = int(round(1e-3 * 2 ** 24))
    dims = wl.dims
    L = dims[0]
    rng = np.random.default_rng(12)
    cand = [0, L - 1, L * L * L - 1, L // 2 + L * (L // 2), 3 * L * L + 7]
    cand += [int(x) for x in rng.integers(0, len(vw), 200)]
    chosen = [v for v in cand if _tie_free(vw, dims, v, k)][:24]
    assert len(chosen) == 24
    one = P.CubicalComplex(cuda(vw.reshape(tuple(reversed(dims)))))
    gmax = float(np.max(np.abs(g)))
    for v in chosen:
        Wpm = []
        for sgn in (1, -1):
            x = vw.copy()
            x[v] += sgn * k
            one.set_weights(cuda(x.reshape(tuple(reversed(dims)))))
            Wpm.append(one.wect(dirs, wl.T, wl.lo, wl.hi).cpu().numpy().astype(object))
        # L+ - L- = (1/N) sum (W+ - W-)(W+ + W- - 2B) * 2^-48, divided by 2 h = 2 k 2^-24
        delta = int(((Wpm[0] - Wpm[1]) * (Wpm[0] + Wpm[1] - 2 * Bk)).sum())
        fd = float(Fraction(delta, 2 * k * N) * Fraction(1, 1 << 24))
        assert abs(fd - float(g[v])) <= 1e-6 * max(abs(float(g[v])), 1e-3 * gmax), (v, fd, float(g[v]))


def test_voxel3d_128_every_direction(P, jobs):
    """The benchmark's step (set_weights + wect) on the 128^3 volume, all 256 directions."""
    wl = S.voxel3d_128()
    grid = cuda(wl.grid)
    cx = P.CubicalComplex(grid)
    out = torch.empty((len(wl.dirs), wl.T), dtype=torch.int64, device=grid.device)
    for _ in range(2):                   # a second step reuses the workspace, as the bench does
        cx.set_weights(grid)
        cx.wect(cuda(wl.dirs), wl.T, wl.lo, wl.hi, out=out)
    got = out.cpu().numpy()
    ref = np.concatenate([j.get() for j in jobs["voxel"]])
    assert np.array_equal(got, ref)
    cx.device_status()


def test_mesh2d_1024_every_tile(P, jobs):
    """1024^2 mesh, default range: the first and last direction of every 32-direction tile."""
    wl = S.mesh2d_1024()
    cx = wl.complex
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(cx.weights), frac_bits=24)
    got = h.wect(cuda(wl.dirs), wl.T).cpu().numpy()
    h.device_status()
    idx = jobs["mesh_idx"]
    ref = np.concatenate([p.get() for p in jobs["mesh"]])
    assert np.array_equal(got[idx], ref)
    assert np.all(got[:, -1] == ref[0, -1])


def test_images2d_4096_every_image(P, jobs):
    """The graph-captured batched launch over all 4096 images, and the per-image loop."""
    wl = S.image_batch()
    dirs = cuda(wl.dirs)
    b = P.CubicalBatch([cuda(x) for x in wl.grids])
    got = b.wect(dirs, wl.T, wl.lo, wl.hi)
    again = b.wect(dirs, wl.T, wl.lo, wl.hi)             # graph replay
    loop = b.wect(dirs, wl.T, wl.lo, wl.hi, loop=True)
    assert torch.equal(got, again) and torch.equal(got, loop)
    got = got.cpu().numpy()
    ref = np.stack([r for j in jobs["images"] for r in j.get()])
    assert np.array_equal(got, ref)


def test_ecf_intensity_paper_sizes(P, jobs):
    """The unweighted ECF of uniform images and volumes, the filter being the intensity, through
    ecf_compute as the benchmark's ECF rows call it."""
    for i, (dims, T) in enumerate(ECF_CASES):
        f = cuda(ecf_filter(dims, 70 + i))
        cx = P.CubicalComplex(None, dims=dims)
        out = torch.empty(10000, dtype=torch.int64, device=f.device)
        got = cx.ecf(f, T, 0.0, 1.0, out=out[:T]).cpu().numpy()
        cx.device_status()
        assert np.array_equal(got, jobs["ecf"][i].get()), (dims, T)
