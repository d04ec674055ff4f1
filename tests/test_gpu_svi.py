"""One SVI step of the lensed-GP model run through the library's kernels
(paper_2105_09465_gb300.svi) against the same step composed from the FP64
oracle (oracle/svi.py), on a small seeded instance."""
import numpy as np
import pytest
import torch

from oracle import svi as osvi
from paper_2105_09465_gb300 import svi, workloads as W
from tests.gpu_util import dev, host, need_gpu
from tests.svi_case import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def close(got, ref, rel, what):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    scale = np.abs(ref).max() + 1e-30
    err = np.max(np.abs(got - ref)) / scale
    assert err <= rel, f"{what}: max error {err:.2e} of max |ref|"


def test_svi_step_matches_the_oracle(orc):
    cfg, guide, data, eps_sp, eps_l = case()
    nx, ny, pix = cfg["pixels"]
    sg = cfg["source_grid"]
    mc = svi.ModelConfig(pixels=W.Grid(nx, ny, 1, pix), source_grid=W.Grid(*sg), sigma_sp=cfg["sigma_sp"],
                         sigma_layers=cfg["sigma_layers"], alpha_sp=cfg["alpha_sp"],
                         alpha_layers=cfg["alpha_layers"], noise=cfg["noise"], gamma=cfg["gamma"],
                         knn_k=cfg["knn_k"])
    gd = svi.Guide(mu=dev(guide["mu"]), L=dev(guide["L"]), C=dev(guide["C"]), sd_sp=dev(guide["sd_sp"]),
                   mu_layers=[dev(a) for a in guide["mu_layers"]], sd_layers=[dev(a) for a in guide["sd_layers"]])
    loss, G = svi.loss_and_grads(mc, gd, dev(data), dev(eps_sp), [dev(e) for e in eps_l])
    g64 = {k: (np.asarray(v, np.float64) if not isinstance(v, list) else [np.asarray(x, np.float64) for x in v])
           for k, v in guide.items()}
    ref, R = osvi.loss_and_grads(orc, cfg, g64, data, eps_sp, eps_l)
    # an FP32 chain (ray-trace, three reductions, windows) against FP64
    assert loss.dtype == torch.float64 and loss.is_cuda
    assert float(loss.item()) == pytest.approx(ref, rel=1e-5)
    close(host(G["d_lens"]), R["d_lens"], 2e-4, "d_lens")
    close(host(G["mu"]), R["mu"], 2e-4, "d_mu")
    close(host(G["L"]), R["L"], 2e-4, "d_L")
    close(host(G["C"]), R["C"], 2e-4, "d_C")
    close(host(G["sd_sp"]), R["sd_sp"], 2e-4, "d_sd_sp")
    close(host(G["layers_mu"][0]), R["layers_mu"][0], 2e-4, "d_mu_layer")
    close(host(G["layers_sd"][0]), R["layers_sd"][0], 2e-4, "d_sd_layer")
