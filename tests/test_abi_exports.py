"""The C-ABI library builds for sm_103a and exports every entry point that
include/dseed.h declares (no GPU needed: nothing is called but version/error)."""
import ctypes
import dataclasses
import os
import re
import subprocess

import pytest

from paper_2410_16727_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "dseed.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dseed_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    try:
        return B.build()
    except RuntimeError as e:  # pragma: no cover - only without a CUDA toolkit
        pytest.skip(str(e))


def test_header_declares_expected_calls():
    names = _declared()
    for want in ("dseed_scene_build_esdf", "dseed_plan_batch", "dseed_cost", "dseed_cost_grad",
                 "dseed_lbfgs_step", "dseed_fk", "dseed_evaluate", "dseed_plan_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(dseed_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version(libpath):
    lib = ctypes.CDLL(libpath)
    lib.dseed_abi_version.restype = ctypes.c_int
    assert lib.dseed_abi_version() == 4
    lib.dseed_last_error.restype = ctypes.c_char_p
    assert lib.dseed_last_error() is not None


def test_host_argument_checks_without_gpu(libpath):
    """Descriptor checks run on the host and need no device."""
    from paper_2410_16727_gb300 import binding as BD
    from paper_2410_16727_gb300 import inputs as I
    BD._lib = None
    lib = BD.load()
    d = BD.plan_desc(1, 1, 300, I.CostParams(), I.OptParams())   # T above the maximum
    n = ctypes.c_size_t()
    assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1
    assert "T = 300" in BD.last_error()
    d = BD.plan_desc(2, 3, 32, I.CostParams(), I.OptParams(iters=5, m=9))
    assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1
    d = BD.plan_desc(2, 3, 32, I.CostParams(), I.OptParams(iters=5, m=5))
    assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == 0
    assert n.value >= 2 * 2 * 3 * 5 * 224 * 4
    for bad in (-1, 9):                                           # swept check: 0..8 interpolants
        d = BD.plan_desc(2, 3, 32, dataclasses.replace(I.CostParams(), n_sweep=bad), I.OptParams())
        assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1
        assert f"n_sweep = {bad}" in BD.last_error()
    d = BD.plan_desc(2, 3, 32, dataclasses.replace(I.CostParams(), n_sweep=8), I.OptParams())
    assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == 0
    # NaN or infinite descriptor entries are refused before any launch
    for field in ("w_c", "eta", "w_R", "w_self"):
        for v in (float("nan"), float("inf")):
            d = BD.plan_desc(2, 3, 32, dataclasses.replace(I.CostParams(), **{field: v}), I.OptParams())
            assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1, (field, v)
            assert "non-finite cost" in BD.last_error()
    d = BD.plan_desc(2, 3, 32, I.CostParams(), I.OptParams(), delta_r=float("nan"))
    assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1
    for field, v, msg in (("c1", float("nan"), "non-finite optimiser"), ("max_step", float("inf"), "non-finite"),
                          ("max_step", 0.0, "max_step"), ("alpha_min", -1e-4, "alpha_min"), ("iters", 0, "iters")):
        d = BD.plan_desc(2, 3, 32, I.CostParams(), dataclasses.replace(I.OptParams(), **{field: v}))
        assert lib.dseed_plan_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == -1, (field, v)
        assert msg in BD.last_error(), (field, BD.last_error())
    r = I.make_robot()
    r.sph_r = r.sph_r.copy()
    r.sph_r[3] = -1.0
    with pytest.raises(BD.DseedError, match="radius"):
        BD.Robot(r)
    h = BD.Robot(I.make_robot())
    assert h.n_spheres == 50
    # Eq. 2 on the robot: argument checks run before any device work
    fk = lib.dseed_nn_fk_mse
    part = ctypes.c_void_p(1)
    assert fk(h.handle, None, None, None, None, 2, 0, 4.0, None, part, 8, None) == -1
    assert "T = 0" in BD.last_error()
    assert fk(h.handle, None, None, None, None, 2, 32, 0.0, None, part, 8, None) == -1
    assert "res_scale" in BD.last_error()
    assert fk(h.handle, None, None, None, None, 2, 32, 4.0, None, part, 2000, None) == -1
    assert "blocks" in BD.last_error()
    assert fk(h.handle, None, None, None, None, 2, 32, 4.0, None, part, 8, None) == -1
    assert "NULL" in BD.last_error()
    assert fk(None, None, None, None, None, 2, 32, 4.0, None, part, 8, None) == -1


def test_conv_tc_descriptor_checks_without_gpu(libpath):
    """The tensor-core convolution validates its descriptor on the host: bad
    shapes or alignment return EINVAL before anything reaches a device."""
    from paper_2410_16727_gb300 import binding as BD
    BD._lib = None
    lib = BD.load()
    fake = 1 << 20                                   # aligned, never dereferenced

    def desc(**kw):
        d = BD.ConvTc()
        d.a0_dev, d.c0, d.n_samples, d.L, d.taps, d.pad = fake, 64, 16, 32, 5, 2
        d.w_dev, d.cout, d.cout_pad, d.out_dev, d.out_ld, d.epilogue = fake, 64, 64, fake, 64, BD.EPI_BF16
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    def rc(d):
        return lib.dseed_nn_conv_tc(ctypes.byref(d), None)

    assert rc(desc(c0=48)) == -1 and "multiples of 64" in BD.last_error()
    assert rc(desc(cout_pad=32, cout=32, out_ld=32)) == -1
    assert rc(desc(L=24)) == -1
    assert rc(desc(taps=9)) == -1
    assert rc(desc(pad=5)) == -1
    assert rc(desc(a0_dev=fake + 4)) == -1 and "aligned" in BD.last_error()
    assert rc(desc(epilogue=BD.EPI_GN)) == -1                       # no bias / gamma / beta
    assert rc(desc(epilogue=BD.EPI_GN, bias_dev=fake, gamma_dev=fake, beta_dev=fake, rows_per_sample=3)) == -1
    assert rc(desc(epilogue=BD.EPI_GN, bias_dev=fake, gamma_dev=fake, beta_dev=fake, rows_per_sample=32,
                   cout=48, out_ld=64)) == -1
    assert lib.dseed_nn_im2col1d_bf16(fake, 4, 8, 7, 3, 1, 1, 8, 24, fake, None) == -1   # C not a multiple of 8


def test_robot_self_pairs_match_the_oracle_without_gpu(libpath):
    """The self-collision pair set is computed on the host when the robot is
    created; it equals the oracle's set, which is computed independently."""
    import numpy as np

    import oracle
    from paper_2410_16727_gb300 import binding as BD
    from paper_2410_16727_gb300 import inputs as I
    BD._lib = None
    robot = I.make_robot()
    mask = BD.Robot(robot).self_pairs()
    spec = I.WORKLOADS["tiny"]
    orc = oracle.Oracle(robot, I.CostParams(), [spec.grid], [np.zeros((0, 6), np.float32)], T=1)
    assert np.array_equal(mask, orc.self_mask)
    assert int(mask.sum()) // 2 == orc.n_self_pairs == 767
    bad = I.make_robot()
    bad.self_margin = float("nan")
    with pytest.raises(BD.DseedError, match="self_margin"):
        BD.Robot(bad)


def test_static_scratch_size_matches_header():
    from paper_2410_16727_gb300 import binding as BD
    text = open(os.path.join(ROOT, "include", "dseed.h")).read()
    m = re.search(r"#define DSEED_STATIC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    assert m and BD.STATIC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


def test_status_codes_match_header():
    from paper_2410_16727_gb300 import binding as BD
    text = open(os.path.join(ROOT, "include", "dseed.h")).read()
    assert int(re.search(r"#define DSEED_ETIMEOUT \((-\d+)\)", text).group(1)) == BD.ETIMEOUT


# ctypes mirror in the binding -> the header's typedef
_STRUCTS = {"RobotDesc": "DseedRobotDesc", "Grid": "DseedGrid", "EsdfJob": "DseedEsdfJob", "Scene": "DseedScene",
            "CostParams": "DseedCostParams", "OptParams": "DseedOptParams", "PlanDesc": "DseedPlanDesc",
            "Problems": "DseedProblems", "LbfgsLayout": "DseedLbfgsLayout", "ServerDesc": "DseedServerDesc",
            "Request": "DseedRequest", "ConvTc": "DseedConvTc", "ServerStats": "DseedServerStats",
            "DeviceInfo": "DseedDeviceInfo"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size of its C typedef and
    each of its fields sits at the C field's offset (a C program built with the
    header prints sizeof / offsetof; a field name missing in C fails to compile)."""
    import shutil

    from paper_2410_16727_gb300 import binding as BD
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda_inc = "/usr/local/cuda/include"
    if cc is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("needs a C compiler and the CUDA runtime header")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dseed.h"', "int main(void) {"]
    want = []
    for py, c in _STRUCTS.items():
        cls = getattr(BD, py)
        lines.append(f'    printf("%zu\\n", sizeof({c}));')
        want.append((f"sizeof {c}", ctypes.sizeof(cls)))
        for name, _ in cls._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({c}, {name}));')
            want.append((f"{c}.{name}", getattr(cls, name).offset))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert len(got) == len(want)
    bad = [(k, w, g) for (k, w), g in zip(want, got) if w != g]
    assert not bad, bad


def _c_kind(param: str) -> str:
    """Coarse kind of one C parameter declaration."""
    p = " ".join(param.replace("\n", " ").split())
    if "*" in p or "cudaStream_t" in p:
        return "ptr"
    words = p.split()
    body = " ".join(w for w in words[:-1] if w not in ("const",)) if len(words) > 1 else p
    return {"int": "int", "float": "float", "double": "double", "size_t": "size_t", "long long": "i64",
            "int64_t": "i64", "unsigned long long": "u64", "uint64_t": "u64"}[body]


def _ctypes_kind(t) -> str:
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    for k, ct in (("int", ctypes.c_int), ("float", ctypes.c_float), ("double", ctypes.c_double),
                  ("size_t", ctypes.c_size_t), ("i64", ctypes.c_longlong), ("u64", ctypes.c_ulonglong)):
        if t is ct:
            return k
    raise AssertionError(f"unexpected ctypes type {t}")


def test_binding_signatures_match_the_header_prototypes():
    """The binding's argument and result types of every entry point agree in
    number and kind (pointer, int, float, double, size_t, 64-bit integer) with
    the header's prototypes, and both name the same entry points."""
    from paper_2410_16727_gb300 import binding as BD
    text = open(os.path.join(ROOT, "include", "dseed.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = {m.group(2): (" ".join(m.group(1).split()), m.group(3))
              for m in re.finditer(r"(int|void|const char \*)\s*\b(dseed_\w+)\s*\(([^;]*?)\)\s*;", text, re.S)}
    assert set(protos) == set(BD._SIGS), set(protos) ^ set(BD._SIGS)
    for name, (ret, params) in protos.items():
        args, res = BD._SIGS[name]
        ps = [p for p in params.split(",") if p.strip() and p.strip() != "void"]
        assert [_c_kind(p) for p in ps] == [_ctypes_kind(a) for a in args], name
        want_res = {"int": ctypes.c_int, "void": None, "const char *": ctypes.c_char_p}[ret]
        assert res is want_res, (name, ret, res)


def test_binding_constants_match_the_header():
    from paper_2410_16727_gb300 import binding as BD
    text = open(os.path.join(ROOT, "include", "dseed.h")).read()
    defs = dict(re.findall(r"#define DSEED_(\w+) \(?(-?[0-9.]+)f?\)?", text))
    for name in ("MAX_SPHERES", "MAX_T", "MAX_HISTORY", "N_METRICS", "ESDF_FAR", "ETIMEOUT"):
        assert float(defs[name]) == float(getattr(BD, name)), name
    # the cost fields the binding fills in order are the header's float fields of DseedCostParams
    body = re.search(r"typedef struct \{([^{}]*)\} DseedCostParams;", re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
                     ).group(1)
    floats = [n.strip() for decl in body.split(";") if decl.strip().startswith("float")
              for n in decl.strip()[len("float"):].split(",")]
    assert tuple(floats) == BD.COST_FIELDS
