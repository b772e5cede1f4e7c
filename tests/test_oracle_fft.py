"""Pins for the oracle's own radix-2 FFT (CPU only).

The split-step of Sec. 3.1 moves between real and reciprocal space with the
discrete Fourier transform; the oracle implements it as an iterative radix-2
FFT.  These tests pin it to the DFT's definition summed by brute force, to an
independent library (numpy.fft), and to Parseval and round-trip identities.
"""
import numpy as np
import pytest

import oracle


def brute_dft(x, sign=-1):
    n = x.size
    j = np.arange(n)
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):                     # plain double loop of the definition
        out[k] = np.sum(x * np.exp(sign * 2j * np.pi * j * k / n))
    return out


def brute_dft2(a, sign=-1):
    ny, nx = a.shape
    out = np.zeros_like(a, dtype=np.complex128)
    ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for ky in range(ny):
        for kx in range(nx):
            out[ky, kx] = np.sum(a * np.exp(sign * 2j * np.pi * (xs * kx / nx + ys * ky / ny)))
    return out


def rand_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1_matches_brute_force(n, sign):
    x = rand_c(n, n)
    ref = brute_dft(x, sign)
    got = oracle.fft1(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(8, 8), (8, 16), (16, 8), (32, 32), (4, 32)])
def test_fft2_matches_brute_force(shape):
    a = rand_c(shape, 7)
    ref = brute_dft2(a, -1)
    got = oracle.fft2(a, -1)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    inv = oracle.fft2(ref, +1)              # inverse carries 1/(nx ny)
    assert np.max(np.abs(inv - a)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("shape", [(64, 128), (256, 32), (512, 512)])
def test_fft2_matches_numpy(shape):
    a = rand_c(shape, 11)
    got = oracle.fft2(a, -1)
    ref = np.fft.fft2(a)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    back = oracle.fft2(got, +1)
    assert np.max(np.abs(back - np.fft.ifft2(ref))) <= 1e-12 * np.max(np.abs(a))


def test_parseval_and_round_trip():
    a = rand_c((128, 64), 3)
    f = oracle.fft2(a, -1)
    assert abs(np.sum(np.abs(f) ** 2) / a.size - np.sum(np.abs(a) ** 2)) <= 1e-10 * np.sum(np.abs(a) ** 2)
    assert np.max(np.abs(oracle.fft2(f, +1) - a)) <= 1e-13 * np.max(np.abs(a)) * 10


def test_single_mode_lands_on_its_bin():
    # a plane wave e^{2 pi i (3 x/nx - 5 y/ny)} transforms to nx*ny at bin (ky=-5, kx=3)
    ny, nx = 16, 32
    ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    a = np.exp(2j * np.pi * (3 * xs / nx - 5 * ys / ny))
    f = oracle.fft2(a, -1)
    expect = np.zeros_like(f)
    expect[ny - 5, 3] = nx * ny
    assert np.max(np.abs(f - expect)) <= 1e-10


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft1(np.ones(12), -1)
    with pytest.raises(ValueError):
        oracle.fft2(np.ones((8, 12)), -1)
