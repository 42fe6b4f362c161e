"""The FP32 predictor's reference-stiffness contractions are written out at build time by
csrc/gen_sref.cpp, with the entries of S^_d (Sec. 4.3, Eq. ader4; transposed for the volume
term, Eq. TAvectors) as instruction immediates.  This test builds and runs the generator
on the host and reads every emitted multiply-add back: the coefficient of acc[m] for the
pre-contracted value (d, j) must be the FP32 rounding of the oracle's exact rational entry
S_d[m][j] (S_d[j][m] for the transposed form; nodes matched by their barycentric
multi-indices, which the generator lists), the entries that vanish exactly must be
absent, the terms of each row must come in increasing (d, j) order, and the column stride
must follow the shared-memory layout rule (16-byte rows, an odd number of 16-byte groups)."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle.refelem import ref_element

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_00619_gb300", "csrc")


@pytest.fixture(scope="module")
def header(tmp_path_factory):
    cxx = os.environ.get("CXX", "g++")
    if shutil.which(cxx) is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("sref")
    exe = str(d / "gen_sref")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(CSRC, "gen_sref.cpp"),
                    os.path.join(CSRC, "refelem.cpp"), "-o", exe], check=True)
    out = str(d / "sref_gen.cuh")
    subprocess.run([exe, out], check=True)
    return open(out).read()


def _struct(text, N):
    a = text.index(f"struct SrefFP32<{N}> {{")
    b = text.index("};", a)
    return text[a:b]


def _node_order(text, N):
    """the generator's lattice-node order as barycentric multi-indices (its header comment)"""
    a = text.index(f"struct SrefFP32<{N}> {{")
    c = text.rindex("// node order", 0, a)
    digits = re.findall(r"\b(\d{4})\b", text[c:a])
    return [tuple(int(ch) for ch in w) for w in digits]


def _terms(body, fname):
    """[(m, kk, coefficient)] of one emitted function, in emission order."""
    a = body.index(f"void {fname}(")
    b = body.index("\n  }\n", a)
    out, base = [], None
    comp = {"x": 0, "y": 1, "z": 2, "w": 3}
    for line in body[a:b].splitlines():
        m = re.search(r"reinterpret_cast<const float4\*>\(b \+ (\d+)\)", line)
        if m:
            base = int(m.group(1))
            continue
        m = re.match(r"\s*acc\[(\d+)\] = fmaf\(([-+0-9a-fx.p]+)f, x\.([xyzw]), acc\[(\d+)\]\);", line)
        if m:
            assert m.group(1) == m.group(4)
            out.append((int(m.group(1)), base + comp[m.group(3)], float.fromhex(m.group(2))))
    return out


def _close_f32(a, b):
    """equal, or one FP32 ulp apart (the generator rounds an extended-precision value)"""
    fa, fb = np.float32(a), np.float32(b)
    return fa == fb or abs(int(fa.view(np.int32)) - int(fb.view(np.int32))) <= 1


@pytest.mark.parametrize("N", [1, 2, 3])
def test_generated_contractions_match_the_exact_stiffness(header, N):
    r = ref_element(N)
    NP = r.Np
    body = _struct(header, N)
    # the product numbers the lattice nodes in its own order: map them onto the oracle's
    order = _node_order(header, N)
    assert sorted(order) == sorted(r.bary) and len(order) == NP
    o = [r.bary.index(a) for a in order]  # product node -> oracle node
    KK = int(re.search(r"KK = (\d+);", body).group(1))
    KKS = int(re.search(r"KKS = (\d+);", body).group(1))
    assert KK == 3 * NP
    assert KKS >= KK and KKS % 4 == 0 and (KKS // 4) % 2 == 1
    for fname, entry in (("contract", lambda d, m, j: r.S_exact[d][o[m]][o[j]]),
                         ("contract_t", lambda d, m, j: r.S_exact[d][o[j]][o[m]])):
        terms = _terms(body, fname)
        got = {}
        for m, kk, c in terms:
            assert (m, kk) not in got, (fname, m, kk)
            got[(m, kk)] = c
        # increasing (d, j) order within each row m
        for m in range(NP):
            kks = [kk for mm, kk, _ in terms if mm == m]
            assert kks == sorted(kks), (fname, m)
        nonzero = 0
        for d in range(3):
            for m in range(NP):
                for j in range(NP):
                    exact = entry(d, m, j)
                    kk = d * NP + j
                    if exact == 0:
                        assert (m, kk) not in got, (fname, d, m, j)
                    else:
                        nonzero += 1
                        assert (m, kk) in got, (fname, d, m, j)
                        assert _close_f32(got[(m, kk)], float(exact)), (fname, d, m, j, got[(m, kk)], float(exact))
        assert len(got) == nonzero
        declared = int(re.search(r"kTerms = (\d+), kTermsT = (\d+);", body).group(1 if fname == "contract" else 2))
        assert declared == nonzero
