"""Delivery-state rendering of dynamic Gaussian scenes on B300 (sm_103a).

Renders a dynamic Gaussian scene as it stands in an incomplete delivery state
and scores it against the complete render, batched over many states, forward
and backward ("Renderable Partial Representations for Dynamic Gaussian
Splatting under Incomplete Delivery", Sections 3-6, Eq. 1, Eq. 3).

* :mod:`.dgs`   -- binding of the C ABI (``include/dgs.h``) of ``libdgs.so``
* :mod:`.synth` -- seeded synthetic scenes, delivery masks, times and cameras
* :mod:`.build` -- nvcc build of ``libdgs.so`` for sm_103a
"""
__all__ = ["dgs", "synth", "build"]
