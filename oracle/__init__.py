"""CPU oracle of the chaos-game hot path (test infrastructure only)."""
