"""A raised loop-nest kernel executes exactly like the textual einsum it
computes: same strategy, same kernel, identical bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402
from oracle import evaluate as ev  # noqa: E402
import workloads as W  # noqa: E402
from test_raise import dg_kernel  # noqa: E402


def test_raised_dg_kernel_matches_textual_einsum_bitwise():
    E = 2000
    D, G, a, b = W.dg_gradient(E=E)
    bufs = {k: torch.from_numpy(v).cuda() for k, v in dict(D=D, G=G, a=a, b=b).items()}
    text = W.dg_gradient_spec(E=E)
    raised = be.raise_kernel(dg_kernel(E, ("el", "dof", "dim", "k"), swap=True))
    outs = {}
    for name, e in (("text", be.Einsum(text)), ("raised", raised)):
        o = [torch.empty((E, 35), dtype=torch.float64, device="cuda") for _ in range(3)]
        be.execute(None, e, bufs, o)
        torch.cuda.synchronize()
        outs[name] = [x.cpu().numpy() for x in o]
    ref = ev.evaluate(text, dict(D=D, G=G, a=a, b=b))
    for x in range(3):
        assert np.array_equal(outs["text"][x], outs["raised"][x])
        assert np.all(np.abs(outs["raised"][x] - ref[x][0]) <= 1e-12 * ref[x][1])
