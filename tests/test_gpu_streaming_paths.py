"""Both code paths of every streaming kernel -- the vectorised one (aligned
buffers, sizes that fill whole vectors) and the general one (buffers offset
from 16-byte alignment, ragged sizes) -- give the oracle's bytes exactly."""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a: np.ndarray, offset: int = 0) -> torch.Tensor:
    """Device copy of `a`, starting `offset` elements into its allocation."""
    flat = torch.from_numpy(np.ascontiguousarray(a).reshape(-1))
    buf = torch.zeros(flat.numel() + offset, dtype=flat.dtype, device="cuda")
    buf[offset:] = flat.cuda()
    return buf[offset:].view(a.shape)


def _empty(shape, dtype, offset: int = 0) -> torch.Tensor:
    n = int(np.prod(shape))
    return torch.empty(n + offset, dtype=dtype, device="cuda")[offset:].view(shape)


SHAPES = [(64, 128), (33, 257), (7, 4), (1, 5), (128, 4100)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("offset", [0, 1])
def test_decode_paths(shape, offset):
    rng = np.random.default_rng(shape[0] + offset)
    q = rng.integers(0, 65536, size=shape, dtype=np.uint16)
    H, W = shape
    dh = _empty(shape, torch.float32, offset)
    awo.awo_decode_u16(_dev(q.view(np.int16), offset), awo.grid(W, H, 1.0), 0.1, dh)
    assert np.array_equal(dh.cpu().numpy(), oracle.decode_u16(q, 0.1))


@pytest.mark.parametrize("shape", SHAPES + [(2, 4), (3, 8)])
@pytest.mark.parametrize("offset", [0, 1])
def test_normals_paths(shape, offset):
    H, W = shape
    rng = np.random.default_rng(H * 3 + W)
    h = (inputs.fbm(max(H, W, 8), 0.8, seed=H + W, relief=700.0)[:H, :W]
         + rng.normal(0, 0.3, size=(H, W))).astype(np.float32)
    g = awo.grid(W, H, 12.5)
    nrm = _empty((3, H, W), torch.float32, offset)
    t2 = _empty((H, W), torch.float32, offset)
    sd = _empty((H, W), torch.float32, offset)
    awo.awo_normals(_dev(h, offset), g, nrm, t2, sd)
    rn, rt, rs = oracle.normals(h, 12.5)
    assert np.array_equal(nrm.cpu().numpy(), rn)
    assert np.array_equal(t2.cpu().numpy(), rt)
    assert np.allclose(sd.cpu().numpy(), rs, rtol=1e-6, atol=1e-5)
    # tan2 only
    t2b = _empty((H, W), torch.float32, offset)
    awo.awo_normals(_dev(h, offset), g, None, t2b, None)
    assert np.array_equal(t2b.cpu().numpy(), rt)


@pytest.mark.parametrize("shape", [(64, 64), (31, 4099), (1, 16), (5, 3)])
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("with_mask", [True, False])
def test_release_paths(shape, offset, with_mask):
    H, W = shape
    rng = np.random.default_rng(H + W + offset)
    t2 = (rng.uniform(0, 1.3, size=(H, W)) ** 2).astype(np.float32)
    g = awo.grid(W, H, 10.0)
    mask = _empty((H, W), torch.uint8, offset) if with_mask else None
    cells = torch.empty(H * W, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    awo.awo_release(_dev(t2, offset), g, 20.0, 40.0, mask, cells, n, ws)
    rm, rc = oracle.release(t2, 20.0, 40.0)
    k = int(n.item())
    assert np.array_equal(cells[:k].cpu().numpy().view(np.uint32), rc)
    if with_mask:
        assert np.array_equal(mask.cpu().numpy(), rm)
    # the same list from the mask
    cells2 = torch.empty(H * W, dtype=torch.int32, device="cuda")
    awo.awo_release_from_mask(_dev(rm, offset), g, cells2, n, ws)
    assert np.array_equal(cells2[:int(n.item())].cpu().numpy().view(np.uint32), rc)


@pytest.mark.parametrize("shape,levels", [((64, 128), 6), ((66, 132), 5), ((33, 257), 5), ((8, 4), 3),
                                          ((2, 8), 3), ((512, 512), 9), ((777, 1000), 11), ((1, 700), 11),
                                          ((130, 2), 8)])
@pytest.mark.parametrize("offset", [0, 1])
def test_finalize_lod_paths(shape, levels, offset):
    H, W = shape
    rng = np.random.default_rng(W + offset)
    cnt = rng.integers(0, 1000, size=(H, W), dtype=np.uint64).astype(np.uint32)
    big = rng.random((H, W)) < 0.2
    cnt[big] = rng.integers(2 ** 30, 2 ** 32, size=int(big.sum()), dtype=np.uint64).astype(np.uint32)
    maxe = rng.uniform(0, 300, size=(H, W)).astype(np.float32)
    maxe[rng.random((H, W)) < 0.3] = 0
    g = awo.grid(W, H, 10.0)
    dv = _empty((H, W), torch.float32, offset)
    awo.awo_finalize(_dev(maxe, offset), g, 9.81, dv)
    vel = oracle.finalize(maxe, 9.81)
    assert np.array_equal(dv.cpu().numpy(), vel)
    shapes = awo.lod_shapes(g, levels)
    cl = [_empty(s, torch.int32, offset) for s in shapes[1:]]
    vl = [_empty(s, torch.float32, offset) for s in shapes[1:]]
    awo.awo_overlay_lod(_dev(cnt.view(np.int32), offset), dv, g, levels, cl, vl)
    rc, rv = oracle.lod(cnt, vel, levels)
    for l in range(1, levels):
        assert np.array_equal(cl[l - 1].cpu().numpy().view(np.uint32), rc[l]), l
        assert np.array_equal(vl[l - 1].cpu().numpy(), rv[l]), l


@pytest.mark.parametrize("shape", [(64, 64), (33, 257), (1, 3)])
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("with_base", [False, True])
def test_compose_paths(shape, offset, with_base):
    H, W = shape
    rng = np.random.default_rng(H * W + offset)
    v = rng.uniform(-5, 80, (H, W)).astype(np.float32)
    v[rng.random((H, W)) < 0.05] = 25.0
    cnt = rng.integers(0, 4, (H, W)).astype(np.uint32)
    base = rng.integers(0, 256, (H, W, 4)).astype(np.uint8) if with_base else None
    g = awo.grid(W, H, 10.0)
    cm = awo.Colormap.make(awo.VELOCITY_STOPS, alpha=0.6, count_min=1)
    out = _empty((H, W, 4), torch.uint8, 4 * offset)
    awo.awo_compose(_dev(v, offset), _dev(cnt.view(np.int32), offset), g, cm,
                    _dev(base, 4 * offset) if with_base else None, out)
    assert np.array_equal(out.cpu().numpy(), oracle.compose(v, cnt, awo.VELOCITY_STOPS, 0.6, 1, base))


@pytest.mark.parametrize("shape", [(64, 64), (33, 257), (1, 3)])
@pytest.mark.parametrize("offset", [0, 1])
def test_snow_paths(shape, offset):
    H, W = shape
    h = inputs.fbm(max(H, W, 8), 0.8, seed=W, relief=2500.0)[:H, :W].astype(np.float32)
    rn, _, _ = oracle.normals(h, 10.0)
    g = awo.grid(W, H, 10.0)
    a = _empty((H, W), torch.float32, offset)
    rgba = _empty((H, W, 4), torch.uint8, 4 * offset)
    awo.awo_snow_cover(_dev(h, offset), _dev(rn[2], offset), g, awo.SnowParams(1200.0, 400.0, 35.0, 6.0), a, rgba)
    ra, rrgba = oracle.snow_cover(h, rn[2], 1200.0, 400.0, 35.0, 6.0)
    assert np.array_equal(a.cpu().numpy(), ra)
    assert np.array_equal(rgba.cpu().numpy(), rrgba)


@pytest.mark.parametrize("shape,levels", [((64, 128), 6), ((33, 257), 5), ((777, 1000), 11), ((1, 700), 11),
                                          ((130, 2), 8), ((5, 3), 1)])
@pytest.mark.parametrize("offset", [0, 1])
def test_finalize_lod_one_pass(shape, levels, offset):
    """awo_finalize_lod equals the oracle's velocity and mipmap (and so
    awo_finalize followed by awo_overlay_lod), also writing the velocity over
    the maximum energy in place."""
    H, W = shape
    rng = np.random.default_rng(H * 7 + W + offset)
    cnt = rng.integers(0, 1000, size=(H, W), dtype=np.uint64).astype(np.uint32)
    cnt[rng.random((H, W)) < 0.1] = 0xFFFFFFF0
    maxe = rng.uniform(0, 300, size=(H, W)).astype(np.float32)
    maxe[rng.random((H, W)) < 0.3] = 0
    g = awo.grid(W, H, 10.0)
    vel = oracle.finalize(maxe, 9.81)
    rc, rv = oracle.lod(cnt, vel, levels)
    shapes = awo.lod_shapes(g, levels)
    for in_place in (False, True):
        dm = _dev(maxe, offset)
        dv = dm if in_place else _empty((H, W), torch.float32, offset)
        cl = [_empty(s, torch.int32, offset) for s in shapes[1:]]
        vl = [_empty(s, torch.float32, offset) for s in shapes[1:]]
        awo.awo_finalize_lod(dm, _dev(cnt.view(np.int32), offset), g, 9.81, levels, dv, cl, vl)
        assert np.array_equal(dv.cpu().numpy(), vel)
        for l in range(1, levels):
            assert np.array_equal(cl[l - 1].cpu().numpy().view(np.uint32), rc[l]), l
            assert np.array_equal(vl[l - 1].cpu().numpy(), rv[l]), l


@pytest.mark.parametrize("shape", SHAPES + [(2, 4), (3, 8)])
@pytest.mark.parametrize("offset", [0, 1])
def test_normals_u16_one_pass(shape, offset):
    """awo_normals_u16 writes the decoded heights and the normals of
    awo_decode_u16 followed by awo_normals, on both paths."""
    H, W = shape
    rng = np.random.default_rng(H * 5 + W + offset)
    q = rng.integers(0, 30000, size=shape, dtype=np.uint16)
    g = awo.grid(W, H, 12.5)
    h = oracle.decode_u16(q, 0.1)
    rn, rt, rs = oracle.normals(h, 12.5)
    dh = _empty((H, W), torch.float32, offset)
    nrm = _empty((3, H, W), torch.float32, offset)
    t2 = _empty((H, W), torch.float32, offset)
    sd = _empty((H, W), torch.float32, offset)
    awo.awo_normals_u16(_dev(q.view(np.int16), offset), g, 0.1, dh, nrm, t2, sd)
    assert np.array_equal(dh.cpu().numpy(), h)
    assert np.array_equal(nrm.cpu().numpy(), rn)
    assert np.array_equal(t2.cpu().numpy(), rt)
    assert np.allclose(sd.cpu().numpy(), rs, rtol=1e-6, atol=1e-5)
    # tan2 only, and no output (decode alone)
    dh2, t2b = _empty((H, W), torch.float32, offset), _empty((H, W), torch.float32, offset)
    awo.awo_normals_u16(_dev(q.view(np.int16), offset), g, 0.1, dh2, None, t2b, None)
    assert np.array_equal(dh2.cpu().numpy(), h) and np.array_equal(t2b.cpu().numpy(), rt)
    dh3 = _empty((H, W), torch.float32, offset)
    awo.awo_normals_u16(_dev(q.view(np.int16), offset), g, 0.1, dh3, None, None, None)
    assert np.array_equal(dh3.cpu().numpy(), h)
