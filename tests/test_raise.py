"""RaiseToBatchedEinsum (be_raise, the first step of Alg. 2): loop-nest
kernels are read back as functional batched einsums whose normal forms,
database keys and name maps equal those of the textual specs they compute."""
import json
import os

import pytest

import paper_2601_12220_b300 as be
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_listing_raises_to_the_paper_einsum():
    g = golden("raise_listing.json")
    e = be.raise_kernel(g["kernel"])
    assert e.outputs == ["y1", "y2"]
    assert e.loop_names == {"a": "i0", "b": "i1"}
    spec = golden("einsum_examples.json")["feinsum_listing"]["spec"]
    assert e.canonicalize().key == be.Einsum(spec).canonicalize().key
    # Alg. 2: the reference's names in the kernel's names
    assert be.identify_kernel(be.Einsum(g["ref_spec"]), e) == g["expected_sigma"]


def dg_kernel(E, loops=("e", "i", "r", "j"), swap=False):
    e, i, r, j = loops
    rows = []
    for x in range(3):
        fac = [f"D[{r},{i},{j}]", f"g{x}({e},{r})", f"U({e},{j})"]
        if swap and x == 1:
            fac = fac[::-1]
        rows.append(f"    R{x}[{e},{i}] = sum([{r},{j}], {'*'.join(fac)})")
    return "\n".join([
        f"{{ [{e},{i},{r},{j}] : 0<={e}<{E} and 0<={i}<35 and 0<={r}<3 and 0<={j}<35 }}",
        "D:f64[3,35,35]", f"G:f64[{E},3,3]", f"a:f64[{E},35]", f"b:f64[{E},35]",
        "g0(p,q) := G[p,q,0]", "g1(p,q) := G[p,q,1]", "g2(p,q) := G[p,q,2]",
        "U(p,q) := sin(a[p,q])*b[p,q]",
        f"for {e}", f"  for {i}", *rows, "  end", "end"])


@pytest.mark.parametrize("loops,swap", [(("e", "i", "r", "j"), False), (("el", "dof", "dim", "k"), True)])
def test_dg_gradient_kernel(loops, swap):
    """The DG gradient as a loop nest (any loop names, factors in any order
    per statement) raises to the gradient's normal form and plans as the
    element strategy."""
    E = 1024
    e = be.raise_kernel(dg_kernel(E, loops, swap))
    text = W.dg_gradient_spec(E=E)
    assert e.canonicalize().key == be.Einsum(text).canonicalize().key
    assert set(e.loop_names.values()) == set(loops)
    assert be.plan_strategy(None, e) == be.STRAT_ELEMENT


def test_lookup_transfers_to_raised_kernel(tmp_path):
    """A configuration recorded for the textual einsum is found for the
    raised kernel: both have one key."""
    E = 512
    ctx = be.Context(str(tmp_path / "db.txt"), device_name="dev", device=-1)
    cfg = be.make_config(be.STRAT_ELEMENT, (64, 128, 2))
    ctx.record(be.Einsum(W.dg_gradient_spec(E=E)).canonicalize(), cfg, 1e-3)
    hit = ctx.lookup(be.raise_kernel(dg_kernel(E)).canonicalize())
    assert hit is not None and tuple(hit[0].tile) == (64, 128, 2, 0)


def test_direct_array_factors_and_annotation():
    """Array accesses as factors, and a rule whose parameter no array
    subscript names (its extent comes from the loop it is called with)."""
    k = "\n".join(["{ [i,j,k] : 0<=i<7 and 0<=j<5 and 0<=k<3 }", "A:f64[7,5]", "B:f64[5,3]",
                   "one(p) := 1.0", "for i", " for k", "  C[i,k] = sum([j], A[i,j]*B[j,k]*one(j))", " end", "end"])
    e = be.raise_kernel(k)
    assert e.out_shape == (7, 3) and e.n == 3
    assert "one(p):f64[5]" in e.text


@pytest.mark.parametrize("kernel,code", [
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\nB:f64[4]\nfor i\n y[i] = sum([j], A[i,j]*B[j])\n z[i] = sum([j], A[i,j])\nend",
     be.EINVALID),                                      # rows with different operand counts
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\nB:f64[4]\nfor i\n y[i] = sum([j], A[i,j]*B[j])\n z[i] = sum([j], A[j,i]*B[j])\nend",
     be.EINVALID),                                      # different index structure
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\nfor i\n y[i] = sum([j], A[i,j]*nope(j))\nend", be.EINVALID),
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\ny[i] = sum([j], A[i,j])", be.EINVALID),   # i is not an enclosing loop
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\nfor i\n y[i] = sum([j], A[i,j])", be.EPARSE),   # no end
    ("{ [i,j] : 0<=i<4 and j<4 }\nA:f64[4,4]\nfor i\n y[i] = sum([j], A[i,j])\nend", be.EPARSE),
    ("{ [i,j] : 0<=i<4 and 0<=j<4 }\nA:f64[4,4]\nfor i\n y[i] = A[i,j]\nend", be.EINVALID),   # j neither output nor summed
])
def test_raise_errors(kernel, code):
    with pytest.raises(be.BEError) as ex:
        be.raise_kernel(kernel)
    assert ex.value.code == code


def test_parsed_einsum_has_no_raised_names():
    import ctypes
    e = be.Einsum("ij,j->i | A,B ; A:f64[3,2] ; B:f64[2]")
    need = ctypes.c_size_t(0)
    assert be.lib().be_raised_name(e.handle, 1, 0, None, 0, ctypes.byref(need)) == be.ENOTFOUND


@pytest.mark.parametrize("text,code", [
    ("ij,j->i | A,B ; A:f64[4,3] ; B:f64[3]", be.EPARSE),                  # no '=>'
    ("ij,j->i | A,B ; A:f64[4,3] ; B:f64[3] => 2 32", be.EPARSE),          # too few config fields
    ("ij,j->i | A,B ; A:f64[4,3] ; B:f64[3] => 2 0 0 0 0 1", be.EPARSE),   # stages without the rest
    ("ij,jk->i | A,B ; A:f64[4,3] ; B:f64[3] => 1 0 0 0 0", be.EINVALID),  # reference fails be_parse
])
def test_transform_library_errors_before_timing(text, code):
    """A malformed transform library is refused while it is read, before
    anything is timed (so on any host)."""
    ctx = be.Context(None, device_name="dev", device=-1)
    with pytest.raises(be.BEError) as ex:
        ctx.load_transforms("# header comment\n" + text + "\n")
    assert ex.value.code == code
    assert ctx.db_size() == 0
