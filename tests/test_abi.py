"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/to.h declares (no compute calls: no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "to.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(to\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libto():
    import paper_2602_19699_gb300 as P
    P.build()
    return P


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tocreate_problem", "tosolve_batch", "toget_trajectories", "tosolve_batch_device"):
        assert required in names


def test_library_exports_every_declared_symbol(libto):
    lib = ctypes.CDLL(libto.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(libto.exported_symbols()) == sorted(_declared_functions())


def test_default_options(libto):
    o = libto.to_default_opts()
    assert (o.max_iter, o.n_alpha, o.prec, o.refine) == (100, 16, libto.TO_MIXED, 1)
    assert o.alpha_decay == 0.5 and o.tol_rel == 1e-8 and o.eps_clip == 1e-8


def test_problem_validation_needs_no_gpu(libto):
    """Argument checks happen on the host before any device call."""
    from paper_2602_19699_gb300 import workload as W
    prob = W.planar3(seed=0)
    with pytest.raises(libto.ToError) as e:
        libto.tocreate_problem(prob.sys, prob.params[:10], 400)
    assert e.value.code == libto.TO_ERR_ARG
    bad = prob.params.copy()
    bad[8 + 1] = 0           # first joint turned into Rx: not the planar chain
    with pytest.raises(libto.ToError) as e:
        libto.tocreate_problem(prob.sys, bad, 400)
    assert "Rz" in str(e.value)
    with pytest.raises(libto.ToError):
        libto.tocreate_problem(99, prob.params, 400)


def test_product_path_does_not_touch_the_oracle():
    """The library package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_19699_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.cpp" not in text and "liboracle" not in text, f


@pytest.mark.parametrize("case", ["quad_parent", "quad_axis", "arm7_axis", "quad_foot"])
def test_parser_rejects_other_joint_trees(libto, case):
    # the device model is compiled for one tree per system; anything else is
    # refused by tocreate_problem's parser, before any CUDA call (no GPU needed)
    from paper_2602_19699_gb300 import workload as W
    P = libto
    prob = W.quad(seed=0, with_actor=False) if case.startswith("quad") else W.arm7(seed=0)
    p = prob.params.copy()
    body = lambda i: W.RIGID_HEADER + W.BODY_STRIDE * i
    if case == "quad_parent":
        p[body(9)] = 8              # hip of leg 1 hung from leg 0's calf
    elif case == "quad_axis":
        p[body(7) + 1] = 0          # thigh about x instead of y
    elif case == "arm7_axis":
        p[body(3) + 1] = 2          # joint 3 about z instead of y
    else:
        c = W.rigid_cost_offset(18)
        p[c + 11] = 7               # foot 0 on the thigh
    with pytest.raises(P.ToError) as e:
        P.tocreate_problem(prob.sys, p, 20)
    assert e.value.code == P.TO_ERR_ARG


def _struct_fields(name):
    """Field names, in order, of a typedef struct { ... } name; in include/to.h."""
    src = open(os.path.join(ROOT, "include", "to.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int a, b" / "const double* p" / "size_t n": names after the type
        names = decl.split(None, 1)[1] if not decl.startswith("const ") else decl.split(None, 2)[2]
        for part in names.split(","):
            fields.append(part.strip().lstrip("*").strip())
    return fields


@pytest.mark.parametrize("name", ["to_problem_desc", "to_solver_opts", "to_tune_row"])
def test_binding_structs_mirror_the_header(libto, name):
    """The ctypes structs of the binding list the header's fields in the
    header's order (a drift would silently shift every later field)."""
    py = [f for f, _ in getattr(libto, name)._fields_]
    assert py == _struct_fields(name)
