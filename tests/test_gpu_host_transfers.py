"""Float host transfers (lbm_init_fields_f32, lbm_moments_f32 and their batch forms) give
exactly the double-transfer results: a float field is the same start as its widened
copy, and float moments are the double moments rounded to nearest.  Asynchronous
transfers (lbm_init_fields_async, lbm_moments_async) give the synchronous results."""
import numpy as np
import pytest

from tests import pairs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_float_init_and_moments_match_double_transfers(prec):
    from paper_1211_6932_gb300 import workloads as wl
    c = pairs.case(75, 52, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    rng = np.random.default_rng(3)
    rho = wl.droplet(75, 52, rl, rv, 15.0, 4.0).astype(np.float32)
    ux = (0.01 * rng.uniform(-1, 1, rho.shape)).astype(np.float32)
    with pairs.gpu_lattice(c, prec) as A, pairs.gpu_lattice(c, prec) as B:
        A.init_fields(rho, ux)                                   # float transfer
        B.init_fields(rho.astype(np.float64), ux.astype(np.float64))
        assert np.array_equal(A.get_populations(), B.get_populations())
        A.step(9)
        B.step(9)
        m64 = A.moments()
        m32 = A.moments(dtype=np.float32)
        for k in ("rho", "ux", "uy"):
            assert m32[k].dtype == np.float32
            assert np.array_equal(m32[k], m64[k].astype(np.float32)), k
        out = np.empty((52, 75), dtype=np.float32)
        assert A.moments(out=out) is out and np.array_equal(out, m32["rho"])
        A.check_guards()


def test_batch_float_transfers():
    from paper_1211_6932_gb300 import Batch, Eos, Instance
    from paper_1211_6932_gb300 import workloads as wl
    cs = [pairs.case(64, 40, tr=0.7, sigma=0.114), pairs.case(33, 70, tr=0.8, sigma=0.114)]
    insts, rhos = [], []
    for c in cs:
        rl, rv = pairs.maxwell(c)
        insts.append(Instance(nx=c["nx"], ny=c["ny"], eos=Eos(a=c["a"], T=c["T"]), G=c["G"],
                              sigma=c["sigma"], s=c["s"], rho_l=rl, rho_v=rv))
        rhos.append(wl.droplet(c["nx"], c["ny"], rl, rv, 10.0, 4.0).astype(np.float32))
    b32, b64 = Batch(insts, precision="fp32"), Batch(insts, precision="fp32")
    try:
        for i, r in enumerate(rhos):
            b32.init_fields(i, r)
            b64.init_fields(i, r.astype(np.float64))
        b32.step(5)
        b64.step(5)
        for i in range(len(cs)):
            assert np.array_equal(b32.get_populations(i), b64.get_populations(i))
            m32, m64 = b32.moments(i, dtype=np.float32), b64.moments(i)
            for k in ("rho", "ux", "uy"):
                assert np.array_equal(m32[k], m64[k].astype(np.float32)), (i, k)
        b32.check_guards()
    finally:
        b32.close()
        b64.close()


def _pinned(a):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_async_transfers_equal_synchronous_ones(prec):
    """Three cycles of upload / 70 steps / read-back queued without waiting (page-locked
    buffers; each upload reuses the staging buffer the previous initialisation read) give
    the synchronous calls' fields bit for bit."""
    from paper_1211_6932_gb300 import workloads as wl
    dt = np.float32 if prec == "fp32" else np.float64
    c = pairs.case(75, 52, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    rng = np.random.default_rng(5)
    starts = [(_pinned(wl.droplet(75, 52, rl, rv, r, 4.0).astype(dt)),
               _pinned((0.01 * rng.uniform(-1, 1, (52, 75))).astype(dt))) for r in (12, 15, 18)]
    outs = [[_pinned(np.zeros((52, 75), dt)) for _ in range(3)] for _ in starts]
    with pairs.gpu_lattice(c, prec) as A:
        for (rho, ux), o in zip(starts, outs):
            A.init_fields_async(rho, ux)
            A.step(70)
            A.moments_async(*o)
        A.sync()
        A.check_guards()
    with pairs.gpu_lattice(c, prec) as B:
        for (rho, ux), o in zip(starts, outs):
            B.init_fields(rho, ux)
            B.step(70)
            m = B.moments(dtype=dt)
            for k, a in zip(("rho", "ux", "uy"), o):
                assert np.array_equal(a, m[k]), k


def test_async_read_back_and_invalid_upload():
    """A synchronous read-back queued after an asynchronous one waits for it (each gets the
    state of its own place in the queue); an invalid asynchronous upload is reported by
    the next sync unless a later upload replaced it."""
    from paper_1211_6932_gb300 import LbmError
    from paper_1211_6932_gb300 import workloads as wl
    c = pairs.case(75, 52, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    good = _pinned(wl.droplet(75, 52, rl, rv, 15.0, 4.0).astype(np.float32))
    bad = _pinned(np.full((52, 75), -1.0, np.float32))
    out = _pinned(np.zeros((52, 75), np.float32))
    with pairs.gpu_lattice(c, "fp32") as L:
        L.init_fields(good)
        L.step(10)
        before = L.moments(dtype=np.float32)["rho"]
        L.moments_async(out)
        L.step(3)
        after = L.moments(dtype=np.float32)["rho"]
        L.sync()
        assert np.array_equal(out, before) and not np.array_equal(after, before)
        L.init_fields_async(bad)
        with pytest.raises(LbmError) as e:
            L.sync()
        assert e.value.code == -1
        L.init_fields_async(bad)
        L.init_fields_async(good)
        L.sync()
        L.step(5)
        L.sync()
        with pytest.raises(ValueError):
            L.init_fields_async(good.astype(np.float64))
