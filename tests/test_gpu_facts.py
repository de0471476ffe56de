"""record_facts and the transform library on the device: a configuration
registered against an idealized reference is timed on synthetic operands,
stored under the reference's normal form and retrieved for isomorphic
einsums (raised kernels included)."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402
import workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_record_facts_then_retrieve_for_raised_kernel(tmp_path):
    g = json.load(open(os.path.join(GOLDEN, "raise_listing.json")))
    ctx = be.Context(str(tmp_path / "db.txt"), device=0)
    cfg = be.make_config(be.STRAT_GENERIC)
    sec = ctx.record_facts(be.Einsum(g["ref_spec"]), cfg, warmup=2, reps=5)
    assert sec > 0 and ctx.db_size() == 1
    hit = ctx.lookup(be.raise_kernel(g["kernel"]).canonicalize())
    assert hit is not None and hit[0].strategy == be.STRAT_GENERIC and hit[1] == pytest.approx(sec)
    # the file holds the fact: a new context reads it back
    assert be.Context(str(tmp_path / "db.txt"), device=0).db_size() == 1


def test_transform_library_best_registration_wins(tmp_path):
    E = 4096
    ref = W.dg_gradient_spec(E=E)
    lib_text = "\n".join([
        "# DG gradient, two element variants",
        f"{ref} => {be.STRAT_ELEMENT} 32 128 2 0",
        f"{ref} => {be.STRAT_ELEMENT} 0 0 3 0",
        f"{ref} => {be.STRAT_GENERIC} 0 0 0 0",
    ])
    ctx = be.Context(None, device=0)
    assert ctx.load_transforms(lib_text, warmup=2, reps=5) == 3
    assert ctx.db_size() == 1
    # the stored fact is the fastest of the three; a renamed copy finds it
    renamed = ref.replace("rij,er,ej->ei", "abc,da,dc->db")
    hit = ctx.lookup(be.Einsum(renamed).canonicalize())
    assert hit is not None and hit[0].strategy == be.STRAT_ELEMENT


def test_record_facts_refuses_a_config_that_does_not_fit():
    ctx = be.Context(None, device=0)
    with pytest.raises(be.BEError) as ex:
        ctx.record_facts(be.Einsum(W.dg_gradient_spec(E=256)), be.make_config(be.STRAT_DENSE_SPLIT),
                         precision=be.PREC_SPLIT)
    assert ex.value.code == be.EUNSUPPORTED
    assert ctx.db_size() == 0
