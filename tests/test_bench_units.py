"""The byte counts behind bench.py's roofline figures, at the benchmark size
(16384 sensors, 512 samples, 128x128x256 output, sigma = 2): the minimum
pipeline bytes per forward are g + f + two passes over the spatial spectrum
and the image spectrum (152.6 MB), and the spread and the interpolation each
move the data g once and the oversampled grid once (167.8 MB)."""
import bench


def test_pipeline_minimum_bytes():
    M, Nt, Nx, Ny, Nz = 16384, 512, 128, 128, 256
    g, f = 4 * M * Nt, 4 * Nx * Ny * Nz
    half = Nx * (Ny // 2 + 1)          # columns kept by the real-data symmetry
    spectrum, image_spectrum = 8 * half * Nt, 8 * half * Nz
    expect = g + f + 2 * spectrum + 2 * image_spectrum
    assert bench.pipeline_min_bytes(M, Nt, Nx, Ny, Nz) == expect
    assert abs(expect / 1e6 - 152.6) < 0.05


def test_stage_bytes_of_the_dominant_kernels():
    M, Nt, Nx, Ny, Nz = 16384, 512, 128, 128, 256
    sb = bench.stage_bytes(M, Nt, Nx, Ny, Nz)
    grid = 4 * (2 * Nx) * (2 * Ny) * Nt   # the sigma = 2 grid, float32
    assert sb["ned_spread"] == sb["ned_interp"] == 4 * M * Nt + grid
    assert abs(sb["ned_interp"] / 1e6 - 167.8) < 0.05
    # every forward stage has its adjoint with the same bytes
    for fwd, adj in (("ned_rowfft", "ned_rowifft"), ("ned_colfft", "ned_colfft_adj"), ("ner_fused", "ner_adj"),
                     ("image_x", "image_x_adj"), ("image_y_c2r", "image_y_adj"), ("ned_spread", "ned_interp")):
        assert sb[fwd] == sb[adj], (fwd, adj)
