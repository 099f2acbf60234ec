"""Plain CPU oracle for the enumerative LTL learner (test infrastructure only)."""
