"""Scribble programs of the library's own workloads (the composition language
of Section 3.1, lowered into the fused chain; see ``cfs_compose_scribble``).

``COMPOSED`` writes the composed 2D/3D scene's chain as verses, a stanza and
a poem; the library expands it into the same device code the op list gives,
so both render the same frame."""

COMPOSED = r"""
// a flame of the 2D branch: rotation, swirl, sinusoidal
__verse flame(| float angle = 0.7f;) {
    rotate2(angle);
    swirl();
    sinusoidal();
}

// pinhole camera at distance `dist` along z
__verse camera(| float dist = 3.5f; float focal = 2.0f;) {
    translate3(0.0f, 0.0f, dist);
    perspective(focal, 1e-3f);
}

// a new branch from a fresh copy of the generator's point
__stanza branch() {
    reset();
    __split_stanza();
}

__poem composed() {
    @VCALL flame();
    splat(0);
    @SCALL branch() {
        torus(1.0f, 0.35f);
        rotate3(1.0f, 0);
        @VCALL camera();
        splat(1);
    }
}
"""
