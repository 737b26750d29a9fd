"""Shared helpers of the tests: problems on the GPU and the matching oracle."""
import numpy as np

from oracle import crf, qp
from oracle import permutohedral as P


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def oracle_features(problem):
    fb, fs = crf.features(problem.rgb, *problem.thetas)
    return crf.to_fp32_features(fb), crf.to_fp32_features(fs)


def oracle_crf(problem, mu=None):
    fb, fs = oracle_features(problem)
    k = P.LatticeGaussian([fb, fs], problem.weights)
    return crf.DenseCRF(problem.unaries, k, mu)


def gpu_setup(dcrf, problems, torch):
    """Features on the GPU (step a1) and the two lattices (step a2) of a batch."""
    rgb = np.concatenate([p.rgb.reshape(-1, 3) for p in problems]).astype(np.float32)
    widths = [p.width for p in problems]
    heights = [p.height for p in problems]
    th = problems[0].thetas
    fb, fs = dcrf.dcrf_features(torch.from_numpy(rgb).cuda(), widths, heights, *th)
    off = np.concatenate([[0], np.cumsum([p.n_pixels for p in problems])]).astype(np.int64)
    lb = dcrf.dcrf_lattice_build(fb, off)
    ls = dcrf.dcrf_lattice_build(fs, off)
    phi = torch.from_numpy(np.concatenate([p.unaries for p in problems])).cuda()
    y0 = torch.from_numpy(np.concatenate([p.y0 for p in problems])).cuda()
    return dict(fb=fb, fs=fs, lb=lb, ls=ls, phi=phi, y0=y0, off=off)


# Frank-Wolfe replayed along the GPU's decisions (see tests/test_gpu_fw_parity.py)
TOL_FILTER = {"f32": 1e-4, "f16": 2e-3}   # filter tolerances (relative to the largest entry)
TOL_ENERGY = 1e-3                          # relaxed energies, relative
TOL_COEF = 1e-3                            # A, B, gap: relative to the largest |energy| of the image
TOL_ALPHA = 1e-3                           # step sizes, absolute
TOL_Y = 1e-3                               # y^T per element, absolute


def replay_image(p, y_gpu, rec_gpu, dec, storage, iters):
    """Replays the GPU's decisions in the oracle; returns the measured errors."""
    c = oracle_crf(p)
    bound = 4.0 * TOL_FILTER[storage] * float((c.c_raw + c.kernel.sum_w).max())
    rows = np.arange(c.n)
    stat = {"excess": 0.0, "agree": 0, "total": 0}

    def on_step(t, g, s):
        ex = g[rows, s] - g.min(axis=1)
        stat["excess"] = max(stat["excess"], float(ex.max()))
        stat["agree"] += int(np.sum(s == np.argmin(g, axis=1)))
        stat["total"] += c.n

    y_o, _, rec_o = qp.frank_wolfe(c, p.y0, iters, decisions=dec.astype(np.int64), on_step=on_step)
    escale = np.abs(rec_o[:, 0]).max()
    return {
        "excess_over_bound": stat["excess"] / bound,
        "agree": stat["agree"] / max(1, stat["total"]),
        "energy": float(np.abs(rec_gpu[:, 0] - rec_o[:, 0]).max() / escale),
        "gap": float(np.abs(rec_gpu[:, 1] - rec_o[:, 1]).max() / escale),
        "alpha": float(np.abs(rec_gpu[:, 2] - rec_o[:, 2]).max()),
        "A": float(np.abs(rec_gpu[:, 3] - rec_o[:, 3]).max() / escale),
        "B": float(np.abs(rec_gpu[:, 4] - rec_o[:, 4]).max() / escale),
        "y": float(np.abs(y_gpu.astype(np.float64) - y_o).max()),
        "final_energy": abs(c.s_cvx(y_gpu.astype(np.float64)) - c.s_cvx(y_o)) / abs(c.s_cvx(y_o)),
    }


def check_replay(err, where=""):
    print(f"\n{where}: " + ", ".join(f"{k} {v:.3g}" for k, v in err.items()))
    assert err["excess_over_bound"] <= 1.0, where
    assert err["energy"] <= TOL_ENERGY and err["final_energy"] <= TOL_ENERGY, where
    assert err["gap"] <= TOL_COEF and err["A"] <= TOL_COEF and err["B"] <= TOL_COEF, where
    assert err["alpha"] <= TOL_ALPHA, where
    assert err["y"] <= TOL_Y, where
