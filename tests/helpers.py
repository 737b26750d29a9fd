"""Shared helpers of the tests: problems on the GPU and the matching oracle."""
import numpy as np

from oracle import crf
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
