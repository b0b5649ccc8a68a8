"""FP64 CPU oracle of the Lagrangian transport hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the CUDA
path computes, written in numpy float64 from the paper's description of the
MPTRAC modules (Section 3.2: ``module_advection``, ``module_diffusion_turb``,
``module_diffusion_meso``, ``module_position``; Section 4.3: ``module_timesteps``,
``module_rng_init``, ``generate_random_nums``; Section 3.1: ``read_met``; Section 6:
the particle sorting modules).  The paper prints no formulas for any of these,
so every numeric choice below is a stated reading; each function's docstring
gives the reading it implements.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import anything from here.  The library path never does: it shares
no code, header, table or helper with this package, and neither imports the
other.  Inputs come from the separate ``workloads`` package.

Pinning status (what each function is checked against, other than itself):

* ``philox``       -- Triton's Philox4x32 (interpreter mode, a third-party
                      library) on CPU; counter-bit avalanche; Box-Muller output
                      checked against the normal distribution.
* ``meteo``, ``sedi`` -- trilinear fields reproduced exactly, count sums and hand
                      cells; Sutherland's reference point, the Stokes and slip
                      limits, textbook settling speeds.
* ``met``          -- torch's bfloat16/float16 rounding; the half-ulp error bound;
                      hand-computed codes.
* ``interp``       -- exact reproduction of fields that are trilinear in
                      (lon, lat, p) and linear in t; brute-force corner sums on
                      tiny grids; periodic-seam shift identity.
* ``transport``    -- closed forms (constant zonal wind, solid-body rotation,
                      uniform omega, the steady analytic wind's exact orbit and
                      second-order convergence); diffusion moments; hand BC cases.
* ``sort``         -- sortedness/stability/permutation invariants and hand keys.
* ``surrogate``    -- torch float64 autograd (library) and central differences.
"""
