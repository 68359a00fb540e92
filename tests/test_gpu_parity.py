"""Bit-exact parity of the CUDA path with the CPU oracle (every height, every
exact sum h and sum h^2) on seeded inputs: the plain single-surface workload,
multisurface jobs across N = 1..7, word widths, tile sizes, ragged lane
counts and tiny lattices."""
import pytest

from paper_1605_02620_gb300.inputs import pow2_schedule
from rsos_testlib import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


def test_plain_L64_N1_1000_sweeps():
    # Plain single surface: L = 64, N = 1, int32 heights, 8x8 tiles, seed 1,
    # 1000 sweeps, W^2 at t = 0 and 2^k.
    times = pow2_schedule(1000) + [1000]
    assert_parity(L=64, N=1, S=1, T=8, seed=1, times=times, t_end=1000, lanes=[0])


@pytest.mark.parametrize("L,N,S,T,order,t_end", [
    (64, 1, 64, 8, 0, 60),     # 64-bit lane words
    (64, 2, 64, 8, 0, 40),     # B = 3
    (64, 3, 32, 8, 0, 40),     # 32-bit lane words
    (64, 4, 64, 8, 0, 40),     # B = 4
    (64, 7, 32, 8, 1, 30),     # largest N, fixed phase order
    (48, 5, 96, 8, 0, 20),     # three 32-lane words, L not a power of two
    (40, 1, 5, 8, 0, 30),      # ragged lane count (5 of 32)
    (16, 2, 64, 4, 0, 50),     # 4x4 tiles
    (8, 1, 64, 2, 0, 50),      # 2x2 tiles (1-site sub-tiles)
    (8, 1, 64, 8, 0, 50),      # one tile covers the lattice
    (64, 1, 64, 16, 0, 30),    # 16x16 tiles
    (2, 1, 32, 2, 0, 100),     # smallest lattice
    (96, 6, 128, 8, 0, 12),    # four words, N = 6
])
def test_multisurface_matches_oracle(L, N, S, T, order, t_end):
    times = sorted({0, 1, 2, t_end // 2, t_end})
    assert_parity(L=L, N=N, S=S, T=T, seed=1000 + L + N + S, order=order, times=times, t_end=t_end)


def test_plain_equals_lane0_and_lane_prefix():
    # The stream of lane j does not depend on the job width: S = 1 (plain
    # path) is lane 0, a 32-lane job is lanes 0..31 of a 64-lane job.
    kw = dict(L=64, N=2, T=8, seed=77, times=[0, 5, 10, 20], t_end=20)
    _, p1, p2, _, ph = gpu_run(S=1, height_lanes=[0], **kw)
    _, a1, a2, _, ah = gpu_run(S=32, height_lanes=[0], **kw)
    _, b1, b2, _, bh = gpu_run(S=64, height_lanes=[0], **kw)
    assert (p1[:, 0] == b1[:, 0]).all() and (p2[:, 0] == b2[:, 0]).all()
    assert (a1 == b1[:, :32]).all() and (a2 == b2[:, :32]).all()
    assert (ph[0] == bh[0]).all() and (ah[0] == bh[0]).all()


@pytest.mark.parametrize("N", [1, 2, 4])
def test_step_height_reduced_size(N):
    # Step-height workload (32 surfaces, B = 2, 3, 4 bits) at L = 256.
    assert_parity(L=256, N=N, S=32, T=8, seed=0, times=[0, 1, 3, 10, 25], t_end=25,
                  height_lanes=[0, 17, 31])


def test_long_run_lane_subset():
    # 2000 sweeps at L = 128, 64 surfaces: lanes 0 and 63 against the oracle.
    times = [0, 1, 10, 100, 1000, 2000]
    assert_parity(L=128, N=1, S=64, T=8, seed=5, times=times, t_end=2000, lanes=[0, 63])
