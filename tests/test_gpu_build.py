"""GPU parity of the volume build (splat, Gladstone-Dale + gradient, FP16
packing) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import hh_inputs as hi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_02048_gb300 import hh

    return hh, torch


def _splat_gpu(hh, torch, parts, dims, h):
    nx, ny, nz = dims
    rho = torch.full((nx * ny * nz,), float("nan"), device="cuda")
    hh.hh_splat_density(torch.from_numpy(parts).cuda(), hh.make_grid(dims, h), rho)
    torch.cuda.synchronize()
    return rho.cpu().numpy().astype(np.float64).reshape(nz, ny, nx)


@pytest.mark.parametrize("dims,n,h,margin", [
    ((37, 29, 45), 3000, 2.0, -3.0),   # ragged grid, particles across and outside faces
    ((64, 64, 64), 20000, 2.0, 4.0),   # interior plume-like load
    ((20, 17, 9), 500, 1.3, 0.0),      # non-integer support radius
    ((8, 8, 8), 1, 3.0, 0.0),          # one particle, support larger than the grid
    ((3, 5, 7), 400, 2.0, -3.0),       # grid thinner than the support on every axis
    ((2, 2, 2), 50, 2.0, -2.0),        # smallest grid
])
def test_splat_matches_oracle(gpu, oracle_lib, dims, n, h, margin):
    hh, torch = gpu
    parts = hi.random_particles(n, dims, seed=n, margin=margin)
    got = _splat_gpu(hh, torch, parts, dims, h)
    want = oracle_lib.splat(parts, dims, h)
    # FP32 kernel values and FP32 atomic accumulation in arbitrary order
    assert np.abs(got - want).max() <= 1e-5 * want.max() + 1e-30


@pytest.mark.parametrize("h", [2.0, 1.75])
def test_splat_support_boundaries(gpu, oracle_lib, h):
    """Particles whose support ends exactly on voxel centres (x - 2h - 1/2 an
    integer), on voxel centres and on cell corners, inside and at the faces."""
    hh, torch = gpu
    dims = (19, 16, 13)
    axis = np.concatenate([np.arange(-1, 20) + 0.5, np.arange(-1, 20) * 1.0,
                           np.arange(0, 20) + 0.5 + 2 * h - np.floor(2 * h)])
    rng = np.random.default_rng(11)
    pos = rng.choice(axis, size=(600, 3))
    pos[:, 1] %= 17.0
    pos[:, 2] %= 14.0
    parts = np.concatenate([pos, rng.uniform(0.5, 2.0, (600, 1))], axis=1).astype(np.float32)
    got = _splat_gpu(hh, torch, parts, dims, h)
    want = oracle_lib.splat(parts, dims, h)
    assert np.abs(got - want).max() <= 1e-5 * want.max()


def test_splat_plume_scene(gpu, oracle_lib):
    """The 262,144-particle plume at 1/4 size (64^3, 4096 particles)."""
    hh, torch = gpu
    parts = hi.plume_particles(4096, 64)
    got = _splat_gpu(hh, torch, parts, (64, 64, 64), 2.0)
    want = oracle_lib.splat(parts, (64, 64, 64), 2.0)
    assert np.abs(got - want).max() <= 1e-5 * want.max()


def test_splat_empty_and_far_particles(gpu):
    hh, torch = gpu
    dims = (10, 11, 12)
    got = _splat_gpu(hh, torch, np.zeros((0, 4), np.float32), dims, 2.0)
    assert np.all(got == 0.0)
    far = np.array([[-50, 5, 5, 1], [5, 500, 5, 1], [np.nan, 5, 5, 1], [5, 5, np.inf, 1]],
                   dtype=np.float32)
    got = _splat_gpu(hh, torch, far, dims, 2.0)
    assert np.all(got == 0.0)


def _field_gpu(hh, torch, rho, K, storage):
    nz, ny, nx = rho.shape
    grid = hh.make_grid((nx, ny, nz), 2.0, storage)
    vol = hh.hh_volume_from_density(torch.from_numpy(rho.astype(np.float32).ravel()).cuda(),
                                    grid, K)
    from parity_util import export_volume

    out = export_volume(hh, torch, vol, (nx, ny, nz))
    info = hh.hh_volume_info(vol)
    info["scales"] = hh.hh_volume_scales(vol)
    vol.close()
    return out, info


@pytest.mark.parametrize("dims", [(64, 64, 64), (33, 2, 17), (5, 40, 3), (64, 7, 9), (32, 15, 70)])
def test_field_fp32_matches_oracle(gpu, oracle_lib, dims):
    hh, torch = gpu
    rho = np.random.default_rng(1).uniform(0.0, 2.5, size=dims[::-1]).astype(np.float32)
    K = float(np.float32(hi.K_GD))
    got, info = _field_gpu(hh, torch, rho, K, "fp32")
    want = oracle_lib.index_field(rho.astype(np.float64), K)
    m = np.abs(want[..., 0]).max()
    # dn = fl(K rho): one rounding; g = fl(fl(dn1 - dn0) / 2): at most 3 roundings of max|dn|
    assert np.abs(got[..., 0] - want[..., 0]).max() <= 2.0**-24 * m * 1.01
    assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 3 * 2.0**-24 * m * 1.01
    assert info["s_n"] == 1.0 and info["s_g"] == 1.0 and info["scales"] == (1.0, 1.0)
    # 2x2x2 micro-bricks over the grid and its one-voxel halo, every axis padded to even
    padded = 8 * ((dims[0] + 3) // 2) * ((dims[1] + 3) // 2) * ((dims[2] + 3) // 2)
    assert info["bytes"] == 16 * padded


def test_field_from_given_dn(gpu, oracle_lib):
    """The tiny plain-method scene: dn given on a 64^3 grid (K = 1)."""
    hh, torch = gpu
    dn = hi.plume_dn_grid(64)
    vol = hh.hh_volume_from_dn(torch.from_numpy(dn.ravel()).cuda(),
                               hh.make_grid((64, 64, 64)))
    from parity_util import export_volume

    got = export_volume(hh, torch, vol, (64, 64, 64))
    want = oracle_lib.index_field(dn.astype(np.float64), 1.0)
    m = np.abs(dn).max()
    assert np.all(got[..., 0] == want[..., 0])  # K = 1: dn is copied exactly
    assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 3 * 2.0**-24 * m


def test_field_fp16_quantisation(gpu, oracle_lib):
    """FP16 storage: per channel group s = the smallest power of two with
    max|.| / s <= 16384; every stored value is the nearest half of value / s
    (error <= 2^-11 relative for normal halves, 2^-25 s absolute in the
    subnormal range)."""
    hh, torch = gpu
    parts = hi.plume_particles(8000, 48)
    rho = oracle_lib.splat(parts, (48, 48, 48), 2.0)
    K = float(np.float32(hi.K_GD))
    want = oracle_lib.index_field(rho.astype(np.float32).astype(np.float64), K)
    got, info = _field_gpu(hh, torch, rho, K, "fp16")
    s_n, s_g = info["s_n"], info["s_g"]
    for s, m in ((s_n, np.abs(want[..., 0]).max()), (s_g, np.abs(want[..., 1:]).max())):
        assert np.frexp(s)[0] == 0.5  # a power of two
        assert 8192 * (1 - 1e-6) < m / s <= 16384 * (1 + 1e-6)
    assert info["scales"] == (info["s_n"], info["s_g"])
    assert info["bytes"] == 8 * 8 * 25**3  # 48 voxels + halo = 50 = 25 bricks per axis
    m = np.abs(want[..., 0]).max()
    for c, s in ((0, s_n), (1, s_g), (2, s_g), (3, s_g)):
        err = np.abs(got[..., c] - want[..., c])
        # the FP32 value before quantisation: dn one rounding, g three of max|dn|
        e32 = 2.0**-24 * (np.abs(want[..., c]) if c == 0 else 3 * m)
        bound = (np.maximum((np.abs(want[..., c]) + e32) * 2.0**-11, s * 2.0**-25) * 1.01
                 + e32 + 2.0**-23 * np.abs(want[..., c]))
        assert np.all(err <= bound), (c, float((err / bound).max()))


def test_build_index_field_matches_parts(gpu, oracle_lib):
    """hh_build_index_field == splat then Gladstone-Dale, checked against the
    oracle end to end (oracle splat in FP64, then Eqs. 12-13)."""
    hh, torch = gpu
    dims = (40, 36, 44)
    parts = hi.plume_particles(6000, 36)
    K = float(np.float32(hi.K_GD))
    vol = hh.hh_build_index_field(torch.from_numpy(parts).cuda(), hh.make_grid(dims, 2.0), K)
    from parity_util import export_volume

    got = export_volume(hh, torch, vol, dims)
    want = oracle_lib.index_field(oracle_lib.splat(parts, dims, 2.0), K)
    m = np.abs(want[..., 0]).max()
    assert np.abs(got[..., 0] - want[..., 0]).max() <= 2e-5 * m
    assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 2e-5 * m



@pytest.mark.parametrize("dims,n", [((70, 37, 53), 70000),    # 60 cells
                                    ((1100, 20, 24), 40000),   # 18-voxel cells: 64 along x
                                    ((33, 33, 33), 20000)])    # 27 cells: the scan's scalar path
def test_build_with_particles_binned_by_cell(gpu, oracle_lib, monkeypatch, dims, n):
    """hh_volume_rebuild sorts the particles by cell before the splat when the
    density grid is larger than L2; forced here on small ragged grids (many
    cells, particles in random order, some outside the grid, NaN and inf):
    the volume equals the oracle's Eqs. 12-13 on its splat, as without."""
    hh, torch = gpu
    monkeypatch.setenv("HH_SPLAT_SORT", "1")
    parts = hi.random_particles(n, dims, seed=3, margin=-3.0)
    bad = np.array([[np.nan, 5, 5, 1], [5, np.inf, 5, 1], [-np.inf, 5, 5, 1]], dtype=np.float32)
    K = float(np.float32(hi.K_GD))
    vol = hh.hh_build_index_field(torch.from_numpy(np.concatenate([parts, bad])).cuda(),
                                  hh.make_grid(dims, 2.0), K)
    from parity_util import export_volume

    got = export_volume(hh, torch, vol, dims)
    vol.close()
    want = oracle_lib.index_field(oracle_lib.splat(parts, dims, 2.0), K)
    m = np.abs(want[..., 0]).max()
    assert np.abs(got[..., 0] - want[..., 0]).max() <= 2e-5 * m
    assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 2e-5 * m


@pytest.mark.parametrize("path", ["trace", "batch", "graph", "none"])
def test_rebuild_after_marches_equals_a_fresh_build(gpu, path):
    """Rebuild / march cycles on one volume and one stream (marches through
    hh_trace, a batched launch or its graph, or none): a rebuild from particle
    set B after rebuilds from set A equals a fresh build from B (up to the
    order of the FP32 atomic sums), so nothing of an earlier frame's density
    survives."""
    hh, torch = gpu
    from parity_util import export_volume

    dims = (40, 36, 44)
    K = float(np.float32(hi.K_GD))
    pa = torch.from_numpy(hi.plume_particles(6000, 36, seed=21)).cuda()
    pb = torch.from_numpy(hi.plume_particles(5000, 36, seed=22)).cuda()
    cams = [hi.orbit_camera(dims, 30.0, 10.0, 32, 24)]
    params = hi.params_euler_adaptive(dims, theta_max=1e-5)
    bg = torch.from_numpy(hi.checker_background()).cuda()
    outs = [{"rgb": torch.empty(32 * 24 * 3, device="cuda")}]
    fresh = hh.hh_build_index_field(pb, hh.make_grid(dims, 2.0), K)
    want = export_volume(hh, torch, fresh, dims)
    fresh.close()
    vol = hh.hh_build_index_field(pa, hh.make_grid(dims, 2.0), K)
    batch = hh.hh_batch_create(vol, cams, params, bg, outs) if path in ("batch", "graph") else None
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for rep in range(2):
            hh.hh_volume_rebuild(vol, pa, K, s)
            if path == "trace":
                hh.hh_trace(vol, cams, params, bg, outs, s)
                hh.hh_trace(vol, cams, params, bg, outs, s)  # a second march: nothing left to clear
            elif path == "batch":
                hh.hh_batch_launch(batch, s)
            elif path == "graph":
                hh.hh_batch_launch_graph(batch, s)
                hh.hh_batch_launch_graph(batch, s)
        hh.hh_volume_rebuild(vol, pb, K, s)
    torch.cuda.synchronize()
    got = export_volume(hh, torch, vol, dims)
    m = np.abs(want[..., 0]).max()
    assert np.abs(got - want).max() <= 1e-5 * m
    if batch is not None:
        batch.close()
    vol.close()


def test_rebuild_of_a_volume_built_from_a_density(gpu):
    """A volume built from a given density has no density scratch of its own;
    its first rebuild from particles allocates one, and later rebuilds reuse
    it, with a batched graph replayed in between: each equals a fresh build."""
    hh, torch = gpu
    from parity_util import export_volume

    dims = (24, 20, 28)
    K = float(np.float32(hi.K_GD))
    rho = torch.zeros(24 * 20 * 28, device="cuda")
    vol = hh.hh_volume_from_density(rho, hh.make_grid(dims, 2.0), K)
    cams = [hi.orbit_camera(dims, 0.0, 0.0, 16, 16)]
    params = hi.params_euler_adaptive(dims, theta_max=1e-5)
    bg = torch.from_numpy(hi.checker_background()).cuda()
    outs = [{"rgb": torch.empty(16 * 16 * 3, device="cuda")}]
    batch = hh.hh_batch_create(vol, cams, params, bg, outs)
    s = torch.cuda.Stream()
    parts = torch.from_numpy(hi.plume_particles(3000, 20, seed=5)).cuda()
    with torch.cuda.stream(s):
        hh.hh_batch_launch_graph(batch, s)
        for _ in range(2):
            hh.hh_volume_rebuild(vol, parts, K, s)
            hh.hh_batch_launch_graph(batch, s)
    torch.cuda.synchronize()
    got = export_volume(hh, torch, vol, dims)
    fresh = hh.hh_build_index_field(parts, hh.make_grid(dims, 2.0), K)
    want = export_volume(hh, torch, fresh, dims)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want[..., 0]).max()
    batch.close()
    fresh.close()
    vol.close()
