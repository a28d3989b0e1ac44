"""FP64 CPU oracle for the NeuralPVS hot path (test infrastructure).

This package is test infrastructure. Only the test suite, the smoke check in
``__graft_entry__.smoke`` and the bench's CPU-baseline / reference leg may import, call, link or
execute it. The product path (``paper_2509_24677_gb300``) never imports it and shares no code,
headers, tables or helpers with it; both consume the same seeded inputs from ``npvs_inputs``.

Modules, each citing the paper passage it restates:
  camera      viewcell -> enclosing frustum and slice table (Sec. 3.2, first paragraph)
  froxel      froxelization (FP32 mirror and FP64) and ray-cast ground truth (Sec. 3.2) in C
  interleave  g_d, g_d^-1, active coarse sites (Sec. 3.3, "3D volume-preserving interleaving")
  network     sparse convolutions as masked dense convolutions (SubM3, 2x2x2 and 3x3x3 stride 2 and
              their transposes, 1x1), the networks (Sec. 3.3, Sec. 2.3)
  rulebook    neighbour maps and the stride-2 output sets by dict lookups (Sec. 2.3)
  loss        weighted Dice + repulsive visibility loss (Sec. 3.3), the Adam update on FP32 master
              weights (Sec. 4.2 hyper-parameters), FNR / FPR (Sec. 5.1)

Where the paper is silent or inconsistent, the reading taken is stated in the function's
docstring.
"""
