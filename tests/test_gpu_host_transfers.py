"""Float host transfers (lbm_init_fields_f32, lbm_moments_f32 and their batch forms) give
exactly the double-transfer results: a float field is the same start as its widened
copy, and float moments are the double moments rounded to nearest."""
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
