"""The quality metric (Sec. IV-C): PSNR = 10 log10(1 / MSE) over the full
grid of the [0, 1]-normalised field.  The library's full-grid PSNR must equal
the one recomputed from the evaluated field.  The paper reports that PSNR
over 500,000 uniformly sampled voxel centres (fixed seed) stays within
0.01 dB of the full grid on its datasets; that is a statistical statement
(the relative standard error of the sampled MSE is std(r^2) / (mean(r^2)
sqrt(n)), about 0.01 dB here), so the check is that the sampled value lies
within four of its standard errors and that the standard error is of that
order."""
import numpy as np
import pytest
import torch

from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def refined():
    V = torch.from_numpy(inputs.grf(256, seed=2)).cuda()
    P, _ = gve.gve_allocate(V, 65_536, seed=2)
    st = gve.gve_refine(P, V, iters=20)
    F = gve.gve_evaluate(P, V.shape)
    return V, F, st


def test_full_grid_psnr_matches_evaluated_field(refined):
    V, F, st = refined
    mse = float(((F.double() - V.double()) ** 2).mean().item())
    assert abs(10 * np.log10(1 / mse) - st["psnr_final"]) <= 1e-4


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sampled_psnr_within_its_standard_error(refined, seed):
    V, F, st = refined
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = torch.from_numpy(rng.integers(0, V.numel(), 500_000)).cuda()
    r = F.reshape(-1)[idx].double() - V.reshape(-1)[idx].double()
    r2 = r * r
    mse = float(r2.mean().item())
    se_db = 10 / np.log(10) * float(r2.std().item()) / (mse * np.sqrt(r2.numel()))
    psnr_s = 10 * np.log10(1 / mse)
    assert se_db < 0.02
    assert abs(psnr_s - st["psnr_final"]) <= 4 * se_db


def test_peak_microbenchmarks_run_and_stay_physical():
    """The roofline denominators: FFMA cannot beat one FMA per lane per clock
    (128 lanes per SM at the maximum SM clock), and the SFU ex2 rate is below
    the FFMA rate."""
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    import subprocess
    try:
        mhz = float(subprocess.check_output(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm",
                                             "--format=csv,noheader,nounits"]).decode().split()[0])
    except Exception:
        mhz = 2100.0
    # best of three runs each: the first launches may still see the clock ramping up
    runs = {kind: [gve.gve_peak_bench(kind, it) for _ in range(3)]
            for kind, it in (("ffma", 2000), ("ffma2", 2000), ("ex2", 500))}
    assert all(ms > 0 for r in runs.values() for _, ms in r)
    ffma, ffma2, ex2 = (max(v for v, _ in runs[k]) for k in ("ffma", "ffma2", "ex2"))
    assert 0 < ffma <= 1.02 * sms * 128 * mhz * 1e6
    assert ffma2 > 0.5 * ffma
    assert 0 < ex2 < ffma
