"""COMPASS oracle (test infrastructure only)."""
