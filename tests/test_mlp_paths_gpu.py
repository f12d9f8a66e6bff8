"""Ray-by-ray parity of the learned map's queries beyond the singlet: the
networks trained on the GPU for the 11-surface lens's transmission path, for
one of its ghost paths (the paper keeps one model per path, Sec. 4.2), and
short-trained networks for all 56 paths of the flare workload, each queried
on the GPU and compared with the oracle's FP64 forward of the same trained
parameters (oracle/mlp.py).

Each query is compared ray by ray by tests/mlp_check.py: FP32 to 3e-5 of
each output's standard deviation plus two FP32 ulps, BF16 / FP16 to twice a
first-order bound of the half-precision rounding of the six layers."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp
from paper_2605_04017_gb300 import batch, lt, workloads as w

from mlp_check import check_query

pytestmark = pytest.mark.gpu

WMAX = 0.2421


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    p = w.eleven_surface_lens(oracle_accept)
    return p, lt.Lens(p), w.eleven_rho(p)


def as64(flat, kind):
    return lt.unflat_params(flat, mlp.layer_sizes(kind))


def train(lens, rho, path_id, fit, reg_steps, cls_steps, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    reg, cls = mlp.init_params("reg", r), mlp.init_params("cls", r)
    return lt.Mlp.train(lens, lt.mlp_frame(path_id, rho, WMAX), batch.DeviceRays(fit), lt.flat_params(reg),
                        lt.flat_params(cls), reg_steps=reg_steps, reg_batch=8192, cls_steps=cls_steps,
                        cls_batch=8192, lr=1e-3, lr_decay=0.95, decay_every=500, seed=seed)


def run_query(m, rays, precision):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    m.query(d.inp, d.lam, o.out, len(rays), precision)
    torch.cuda.synchronize()
    return o.numpy()


def check(m, rays, rho, precision, label):
    st = m.stats()
    reg_f, cls_f = m.params()
    out, flags = run_query(m, rays, precision)
    rep = check_query(out, flags, as64(reg_f, "reg"), as64(cls_f, "cls"), rays, rho, WMAX, st["t_mean"],
                      st["t_std"], precision, label)
    print("learned map", label, precision, rep)
    return rep


@pytest.fixture(scope="module")
def eleven_trained(eleven):
    p, lens, rho = eleven
    fit = w.entrance_rays(1 << 19, w.SEED_BASE + 211, rho)
    return {pid: train(lens, rho, pid, fit, 4000, 3000, 20 + pid) for pid in (0, 20)}


@pytest.mark.parametrize("precision", [lt.MLP_F32, lt.MLP_BF16, lt.MLP_F16])
@pytest.mark.parametrize("path_id", [0, 20])
def test_eleven_learned_map_matches_oracle_forward(eleven, eleven_trained, path_id, precision):
    p, lens, rho = eleven
    m = eleven_trained[path_id]
    st = m.stats()
    assert st["n_valid"] > 10000, st
    rays = w.eleven_rays(p, 30000)
    rep = check(m, rays, rho, precision, f"eleven path {path_id}")
    assert rep["compared"] > 1000 and rep["decided"] > 0.9


def test_flare_maps_sampled_against_oracle(eleven):
    """One short-trained map per path of the flare workload (main + 55
    ghosts); each path's BF16 query (the flare workload's map variant) on 512
    rays and its FP32 query on 256, ray by ray against the oracle's forward."""
    p, lens, rho = eleven
    fit = w.entrance_rays(1 << 16, w.SEED_BASE + 212, rho)
    rays = w.flare_rays(p, 512)
    worst, checked = 0.0, 0
    for pid in range(lens.n_paths):
        try:
            m = train(lens, rho, pid, fit, 300, 200, 500 + pid)
        except lt.LTError:
            continue   # fewer than 2 of the uniform training rays traverse the path
        if m.stats()["n_valid"] < 64:
            continue   # too few valid rays for target statistics worth checking
        rep = check(m, rays, rho, lt.MLP_BF16, f"flare path {pid}")
        worst = max(worst, rep.get("pos_err_over_bound", 0.0))
        check(m, rays.subset(slice(0, 256)), rho, lt.MLP_F32, f"flare path {pid}")
        checked += 1
    print("flare maps checked", checked, "worst BF16 position error / bound", worst)
    assert checked >= 50
