"""The C ABI from plain C: tests/c/abi_host.c (host-side entry points only, no
GPU) and tests/c/abi_gpu.c (create, sweep, get_field, get_G, measure on the
GPU) are compiled with gcc against include/afqmc.h, linked to libafqmc.so and
run; the GPU program's field, G and observables are held to the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def compile_c(name, tmp_path):
    from paper_2609_14668_b300 import build
    build.build()
    libdir = os.path.dirname(build.LIB)
    exe = tmp_path / name
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", name + ".c"), "-L", libdir, "-lafqmc",
                    f"-Wl,-rpath,{libdir}", "-lm", "-o", str(exe)], check=True)
    return exe


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_caller(tmp_path):
    exe = compile_c("abi_host", tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert "c abi ok" in r.stdout


@pytest.mark.gpu
@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_gpu_chain_matches_oracle(tmp_path):
    """Two sweeps of an L = 3 chain from plain C, in lockstep with the oracle
    chain of the same seed: same initial field and decisions (fields and
    accepted counts exactly equal), G at slice 0 and its observables to 1e-10."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.dqmc import Model, Chain
    from oracle.observables import measure
    exe = compile_c("abi_gpu", tmp_path)
    out = tmp_path / "chain.bin"
    r = subprocess.run([str(exe), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "c gpu abi ok" in r.stdout
    raw = out.read_bytes()
    N, M = np.frombuffer(raw, np.int32, 2)
    proposed, accepted = np.frombuffer(raw, np.uint64, 2, offset=8)
    off = 24
    field = np.frombuffer(raw, np.int8, M * N, offset=off).reshape(M, N)
    off += M * N
    G = np.frombuffer(raw, np.float64, N * N, offset=off).reshape(N, N)
    obs = np.frombuffer(raw, np.float64, 10, offset=off + 8 * N * N)

    m = Model(3, U=3.73, beta=3.0, dtau=0.1)
    oc = Chain(m, n_delay=4, n_stab=10, seed=2024)
    for _ in range(2):
        oc.sweep()
    assert (N, M) == (m.N, m.M)
    assert proposed == 2 * 2 * m.N * m.M
    assert accepted == oc.accepted
    assert np.array_equal(field, oc.field)
    G_ref = m.green_stable(oc.field, 0, 10)
    assert np.abs(G - G_ref).max() < 1e-10 * np.abs(G_ref).max()
    ref = measure(m, G_ref)
    keys = ("energy", "double_occ", "ekin", "density", "m2", "S_af", "S_af_dk", "R_m2", "Czz_half", "chi_e")
    for k, v in zip(keys, obs):
        assert abs(v - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), (k, v, ref[k])
