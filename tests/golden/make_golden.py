"""Writes the oracle's golden fixtures (``tests/golden/*.json``).

Run from the repository root: ``python tests/golden/make_golden.py``.  Every
value comes from ``oracle/`` on seeded inputs of ``gs2d_inputs`` (no CUDA
code is called).  A fixture stores, per output, its shape, sum, sum of
squares and values at seeded sample positions; ``tests/test_oracle_golden.py``
recomputes them and compares within a relative 1e-12 (OpenMP and BLAS
summation order).  The paper prints no worked example of these functions, so
the fixtures pin the oracle against unnoticed change, not against the paper:
its pins are in ``tests/test_oracle_*.py``.  A change of a stored value needs
a commit message naming the passage, or the reading of it, that justifies it.
"""

from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def summary(a, samples: int = 12, seed: int = 0) -> dict:
    """Shape, sum, sum of squares and seeded samples of an array (float64)."""
    a = np.asarray(a, np.float64)
    flat = a.reshape(-1)
    idx = np.random.Generator(np.random.PCG64(seed)).choice(flat.size, min(samples, flat.size),
                                                            replace=False)
    return {"shape": list(a.shape), "sum": float(flat.sum()), "sumsq": float((flat * flat).sum()),
            "idx": [int(i) for i in idx], "values": [float(flat[i]) for i in idx]}


def fixtures() -> dict:
    """name -> {"cites", "inputs", "outputs"}: what the oracle computes now."""
    import oracle
    from oracle import bitstream, cnn, quant, superpixel
    from gs2d_inputs import (conferencing_frame, random_gaussians, rng, smooth_noise_target)

    oracle.build()
    out = {}

    p = random_gaussians(12, 24, 16, seed=3)
    out["render"] = {
        "cites": "Eq. 2 (Sec. 3.1): alpha blending of the 2D Gaussians, brute force, float64",
        "inputs": "random_gaussians(12, 24, 16, seed=3), 24 x 16",
        "outputs": {"img": summary(oracle.render(p, 24, 16))}}

    target = smooth_noise_target(24, 16, seed=4)
    r = oracle.loss_and_grad(p, target)
    out["loss_grad"] = {
        "cites": "Eq. 2 and its gradient with respect to the parameters of Eq. 1 (Sec. 3.1), "
                 "L2 loss",
        "inputs": "random_gaussians(12, 24, 16, seed=3) against smooth_noise_target(24, 16, seed=4)",
        "outputs": {"loss": summary([r["loss"]]), "grad": summary(r["grad"], 18, 1)}}

    g = rng(7)
    x = cnn.bf16_round(g.normal(size=(1, 9, 10, 8)))
    w = cnn.bf16_round(g.normal(size=(16, 73)) / 8.0)
    out["conv"] = {
        "cites": "Sec. 3.2 B: a 3 x 3 stride-2 convolution of the learned initialiser, bias as "
                 "the last weight column",
        "inputs": "x = bf16(normal(1, 9, 10, 8)), w = bf16(normal(16, 73) / 8), rng(7)",
        "outputs": {"z": summary(cnn.conv(x, w, 3, 2, 1), 16, 2)}}

    q = random_gaussians(40, 64, 48, seed=8)
    bits = [quant.HALF, quant.HALF, 6, 6, 6, 8, 8, 8, 0]
    codes, values, ranges = quant.quantize(q, bits, refine=True)
    out["quantize"] = {
        "cites": "Sec. 3.3 A: per-attribute quantisation (half-precision means, uniform "
                 "Cholesky and colour codes over each row's range)",
        "inputs": "random_gaussians(40, 64, 48, seed=8), bits [half, half, 6, 6, 6, 8, 8, 8, 0]",
        "outputs": {"codes": summary(codes, 16, 3), "values": summary(values, 16, 4),
                    "ranges": summary(ranges, 8, 5)}}

    frame, mask = conferencing_frame(64, 48, seed=9)
    gb = rng(10)
    bg_xy = np.stack([gb.uniform(0, 64, 60), gb.uniform(0, 48, 60)], axis=1)
    params, info = superpixel.roi_init(frame, mask, 60, 0.7, bg_xy)
    out["roi_init"] = {
        "cites": "Sec. 3.2 A: K-means superpixels of the ROI, one Gaussian per segment from its "
                 "pixel moments, background Gaussians at given positions",
        "inputs": "conferencing_frame(64, 48, seed=9), n 60, roi_frac 0.7, background positions "
                  "uniform from rng(10)",
        "outputs": {"params": summary(params, 18, 6), "M": summary([info["M"]])}}

    counts = [200, 9, 11, 10, 200, 8, 12]
    payload = [9000.0, 610.0, 700.0, 655.0, 8800.0, 540.0, 780.0]
    sb = bitstream.sequence_bits(counts, payload, 4)
    out["sequence_bits"] = {
        "cites": "Eq. 3-4 (Sec. 3.3 B): I-frame bits plus P-frame bits less the bits-back saving",
        "inputs": "counts [200, 9, 11, 10, 200, 8, 12], payload bits as stored, GOP 4",
        "outputs": {"bits": summary([sb["i_bits"], sb["p_bits"], sb["savings"],
                                     sb["total_bits"], sb["i_frames"], sb["p_frames"]], 6, 7)}}
    return out


def main():
    for name, fx in fixtures().items():
        path = os.path.join(HERE, name + ".json")
        with open(path, "w") as f:
            json.dump(fx, f, indent=1, sort_keys=True)
            f.write("\n")
        print("wrote", os.path.relpath(path, ROOT))


if __name__ == "__main__":
    main()
