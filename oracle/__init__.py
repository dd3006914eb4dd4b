"""Oracle: a plain, slow CPU reference for the AIM-accelerated SIE operators.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2003_11679_gb300``)
and never imports it.

Modules (each function cites the passage of Sharma & Triverio, "An accelerated
surface integral equation method for the electromagnetic modeling of
dielectric and lossy objects of arbitrary conductivity", that it follows):

* ``rwg``    -- RWG edge table of a closed triangle mesh (Sec. II-A).
* ``mom``    -- dense Galerkin matrices of Eqs. (opL), (opK) and the identity
                operator I_x, in FP64 (C kernel ``mom.c`` + numpy assembly).
* ``aim``    -- the AIM decomposition of Eqs. (AIM_Lin)/(AIM_Kin): grid,
                projection/interpolation by moment matching, grid convolution
                (direct sum and FFT), near-region correction (Eqs. LinNRP/KinNRP).
* ``bounds`` -- the Lagrange interpolation error bound of Eqs. (Lbounds)-(Ddef).
* ``mie``    -- Mie series of a homogeneous sphere (the paper's RCS check).
* ``system`` -- the dense and AIM forms of Eqs. (GIBCsys) and (sys),
                plane-wave excitation, RCS, SIBC, several objects.
* ``ports``  -- delta-gap ports, admittance and S parameters (Secs. II, V),
                radiated and absorbed power.
* ``dual``   -- dual (Buffa-Christiansen) basis on the barycentric
                refinement (Sec. V discussion).

Parity status of each function is stated in its docstring; a function with
no independent pin says "parity unpinned".
"""
